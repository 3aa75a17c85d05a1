"""Python binding of the C ABI in include/gh.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libgh.so``; this module
allocates device buffers with torch, passes raw pointers and the current
torch stream, and wraps the results.  There is no fallback: if the library is
missing or the GPU is not an sm_103 device, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _buildlib

GH_OK, GH_ERR_ARG, GH_ERR_CAPACITY, GH_ERR_CUDA, GH_ERR_NONFINITE, GH_ERR_UNIMPLEMENTED, GH_ERR_DEVICE = range(7)
GH_SDB_CSG, GH_SDB_MLP = 0, 1
GH_FP32, GH_BF16_REFINE, GH_BF16_REFINE_X6 = 0, 1, 2
GH_TAU_DIAGONAL, GH_TAU_HALF_DIAGONAL = 0, 1
PRECISIONS = {"fp32": GH_FP32, "bf16": GH_BF16_REFINE, "bf16_refine": GH_BF16_REFINE, "bf16x6": GH_BF16_REFINE_X6}
GH_METHOD_HOP, GH_METHOD_ENUM = 0, 1
METHODS = {"hop": GH_METHOD_HOP, "enum": GH_METHOD_ENUM}

_lock = threading.Lock()
_lib = None


class GhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gh error %d: %s" % (code, msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class SdbDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("blob", ctypes.c_void_p), ("blob_bytes", ctypes.c_size_t),
                ("lipschitz_scale", ctypes.c_float)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tau_mode", ctypes.c_int32), ("eps", ctypes.c_float),
                ("sync", ctypes.c_int32), ("ray_block", ctypes.c_int32), ("mlp_tiles", ctypes.c_int32),
                ("method", ctypes.c_int32)]


STAT_FIELDS = ["status", "columns", "hop_evals", "marked_cells", "unique_vertices", "refined_vertices",
               "surface_cells", "triangles", "row_slots", "mesh_vertices"]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in STAT_FIELDS] + [("reserved", ctypes.c_int64 * 6)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("tri_xyz", ctypes.c_void_p), ("tri_keys", ctypes.c_void_p), ("capacity_tris", ctypes.c_int64),
                ("n_tris", ctypes.c_void_p), ("cell_ids", ctypes.c_void_p), ("cell_cases", ctypes.c_void_p),
                ("capacity_cells", ctypes.c_int64), ("n_cells", ctypes.c_void_p), ("stats", ctypes.c_void_p),
                ("vert_xyz", ctypes.c_void_p), ("tri_idx", ctypes.c_void_p), ("capacity_verts", ctypes.c_int64),
                ("n_verts", ctypes.c_void_p)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("n_phases", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms", ctypes.c_double * 8)]


PHASES = ["hop", "lists", "vertices", "select", "refine", "mc"]


def lib_path() -> str:
    return _buildlib.LIB


def lib():
    """Loads libgh.so, building it first when nvcc is available."""
    global _lib
    with _lock:
        if _lib is None:
            if not _buildlib.up_to_date():
                _buildlib.build_library()
            if not os.path.exists(_buildlib.LIB):
                raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build()" % _buildlib.LIB)
            L = ctypes.CDLL(_buildlib.LIB)
            P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            sig = {
                "gh_create_sdb": (ctypes.c_int, [ctypes.POINTER(SdbDesc), ctypes.POINTER(P)]),
                "gh_destroy_sdb": (ctypes.c_int, [P]),
                "gh_sdb_calibrate": (ctypes.c_int, [P, ctypes.POINTER(Grid), I64, ctypes.c_uint64,
                                                    ctypes.POINTER(ctypes.c_float), P]),
                "gh_polygonize": (ctypes.c_int, [ctypes.POINTER(Grid), P, ctypes.POINTER(Options),
                                                 ctypes.POINTER(MeshDesc), P]),
                "gh_polygonize_batch": (ctypes.c_int, [ctypes.c_int, P, P, ctypes.POINTER(Options), P, P, P]),
                "gh_batch_graph_launch": (ctypes.c_int, [P, P]),
                "gh_batch_graph_free": (ctypes.c_int, [P]),
                "gh_backward": (ctypes.c_int, [P, P, P, I64, P, P]),
                "gh_eval": (ctypes.c_int, [P, P, I64, P, I32, P]),
                "gh_mc_table": (ctypes.c_int, [P, P]),
                "gh_mlp_param_count": (I64, [I32, I32]),
                "gh_last_error": (ctypes.c_char_p, []),
                "gh_version": (ctypes.c_char_p, []),
                "gh_set_profiling": (ctypes.c_int, [ctypes.c_int]),
                "gh_polygonize_csg_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), P, I32, I32,
                                                             ctypes.POINTER(MeshDesc), P]),
                "gh_last_profile": (ctypes.c_int, [ctypes.POINTER(Profile)]),
                "gh_release_cache": (ctypes.c_int, []),
                "gh_column_order": (I64, [I32, I64]),
                "gh_set_wait_limit_ns": (ctypes.c_int, [ctypes.c_uint64]),
                "gh_polygonize_cont": (ctypes.c_int, [ctypes.POINTER(Grid), P, P, I32, ctypes.POINTER(Options),
                                                      ctypes.POINTER(MeshDesc), P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    """Names declared in include/gh.h that the library must export."""
    return ["gh_create_sdb", "gh_destroy_sdb", "gh_sdb_calibrate", "gh_polygonize", "gh_polygonize_batch",
            "gh_backward", "gh_eval", "gh_mc_table", "gh_mlp_param_count", "gh_last_error", "gh_version",
            "gh_set_profiling", "gh_last_profile", "gh_polygonize_csg_noalloc", "gh_batch_graph_launch",
            "gh_batch_graph_free", "gh_release_cache", "gh_column_order", "gh_polygonize_cont",
            "gh_set_wait_limit_ns"]


def check(rc):
    if rc != GH_OK:
        raise GhError(rc, lib().gh_last_error().decode())


def mc_table():
    """The library's Marching Cubes table (host-side, no GPU needed)."""
    ntri = np.zeros(256, np.int32)
    edges = np.zeros((256, 5, 3), np.int32)
    check(lib().gh_mc_table(ntri.ctypes.data, edges.ctypes.data))
    return ntri, edges


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _grid(N, lo, hi) -> Grid:
    lo3 = np.broadcast_to(np.asarray(lo, np.float32), (3,))
    hi3 = np.broadcast_to(np.asarray(hi, np.float32), (3,))
    g = Grid()
    g.N = int(N)
    for a in range(3):
        g.lo[a] = float(lo3[a])
        g.hi[a] = float(hi3[a])
    return g


# ---------------------------------------------------------------------------
# SDB objects
# ---------------------------------------------------------------------------
class Sdb:
    kind = None

    def __init__(self, blob: bytes, lam: float = 1.0):
        self._blob = ctypes.create_string_buffer(blob, len(blob))
        d = SdbDesc(self.kind, ctypes.cast(self._blob, ctypes.c_void_p), len(blob), float(lam))
        h = ctypes.c_void_p()
        check(lib().gh_create_sdb(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.lam = float(lam)
        self._cap = {}

    def close(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.gh_destroy_sdb(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csg_blob(prims) -> bytes:
    """prims: [n, 17] rows (type, op, centre[3], param[3], rot[9]) -> CSG blob."""
    p = np.asarray(prims, np.float64).reshape(-1, 17)
    rec = np.zeros(p.shape[0], dtype=[("type", "<i4"), ("op", "<i4"), ("c", "<f4", 3), ("p", "<f4", 3),
                                      ("rot", "<f4", 9), ("pad", "<f4", 3)])
    rec["type"] = p[:, 0].astype(np.int32)
    rec["op"] = p[:, 1].astype(np.int32)
    rec["c"] = p[:, 2:5]
    rec["p"] = p[:, 5:8]
    rec["rot"] = p[:, 8:17]
    hdr = np.array([p.shape[0], 0, 0, 0], np.int32)
    return hdr.tobytes() + rec.tobytes()


def paper_mlp(params, width, n_mid, lam=1.5) -> "MlpSdb":
    """A network in the paper's form (Sec. 5.2): SDB = network / lambda, no
    radial term, batch normalisation already folded into the weights."""
    return MlpSdb(params, width, n_mid, r0=0.0, alpha=1.0, beta=1.0, lam=lam, radial=False)


class CsgSdb(Sdb):
    kind = GH_SDB_CSG

    def __init__(self, prims):
        self.prims = np.asarray(prims, np.float64).reshape(-1, 17)
        super().__init__(csg_blob(self.prims), 1.0)


GH_MLP_NO_RADIAL = 1


def mlp_blob(params, width, n_mid, r0, alpha, beta, radial=True) -> bytes:
    p = np.ascontiguousarray(params, np.float32).ravel()
    flags = 0 if radial else GH_MLP_NO_RADIAL
    hdr = np.array([width, n_mid, flags, 0], np.int32).tobytes() + np.array([r0, alpha, beta, 0], np.float32).tobytes()
    return hdr + p.tobytes()


class MlpSdb(Sdb):
    kind = GH_SDB_MLP

    def __init__(self, params, width, n_mid=5, r0=0.6, alpha=0.1, beta=1.1, lam=1.0, radial=True):
        self.params = np.ascontiguousarray(params, np.float32).ravel()
        self.width, self.n_mid = int(width), int(n_mid)
        self.r0, self.alpha, self.beta = float(r0), float(alpha), float(beta)
        self.radial = bool(radial)
        n = int(lib().gh_mlp_param_count(self.width, self.n_mid))
        if self.params.size != n:
            raise ValueError("expected %d parameters, got %d" % (n, self.params.size))
        super().__init__(mlp_blob(self.params, width, n_mid, r0, alpha, beta, radial), lam)
        self.eps = None

    def calibrate(self, N=1024, lo=-1.0, hi=1.0, n_points=1 << 20, seed=0, stream=None) -> float:
        e = ctypes.c_float()
        g = _grid(N, lo, hi)
        check(lib().gh_sdb_calibrate(self.handle, ctypes.byref(g), int(n_points), int(seed), ctypes.byref(e),
                                     _stream_ptr(stream)))
        self.eps = float(e.value)
        return self.eps


# ---------------------------------------------------------------------------
# polygonization
# ---------------------------------------------------------------------------
class Mesh:
    """Triangle soup on the device: tri_xyz [T,3,3] float32, tri_keys [T,3]
    int64 edge keys (optional), surface cells (optional), statistics, and
    (indexed=True) the indexed mesh: verts [V,3] float32 and faces [T,3] int32
    into them, in the soup's triangle order."""

    def __init__(self, tri_xyz, tri_keys, cell_ids, cell_cases, stats, verts=None, faces=None):
        self.tri_xyz = tri_xyz
        self.tri_keys = tri_keys
        self.cell_ids = cell_ids
        self.cell_cases = cell_cases
        self.stats = stats
        self.verts = verts
        self.faces = faces

    @property
    def n_tris(self):
        return int(self.tri_xyz.shape[0])


class Buffers:
    """Caller-owned device buffers of one polygonization (reusable)."""

    def __init__(self, cap_tris, keys=False, cap_cells=0, device=None, cap_verts=0):
        import torch

        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.cap_tris = int(cap_tris)
        self.cap_cells = int(cap_cells)
        self.cap_verts = int(cap_verts)
        if cap_verts:
            keys = True  # the face indices are derived from the edge keys
        self.tri_xyz = torch.empty((max(self.cap_tris, 1), 3, 3), dtype=torch.float32, device=dev)
        self.tri_keys = torch.empty((max(self.cap_tris, 1), 3), dtype=torch.int64, device=dev) if keys else None
        self.cell_ids = torch.empty(max(self.cap_cells, 1), dtype=torch.int64, device=dev) if cap_cells else None
        self.cell_cases = torch.empty(max(self.cap_cells, 1), dtype=torch.uint8, device=dev) if cap_cells else None
        self.verts = torch.empty((max(self.cap_verts, 1), 3), dtype=torch.float32, device=dev) if cap_verts else None
        self.faces = torch.empty((max(self.cap_tris, 1), 3), dtype=torch.int32, device=dev) if cap_verts else None
        self.counts = torch.zeros(3, dtype=torch.int64, device=dev)  # n_tris, n_cells, n_verts
        self.stats = torch.zeros(16, dtype=torch.int64, device=dev)
        self.desc = MeshDesc()
        d = self.desc
        d.tri_xyz = self.tri_xyz.data_ptr()
        d.tri_keys = self.tri_keys.data_ptr() if keys else None
        d.capacity_tris = self.cap_tris
        d.n_tris = self.counts.data_ptr()
        d.cell_ids = self.cell_ids.data_ptr() if cap_cells else None
        d.cell_cases = self.cell_cases.data_ptr() if cap_cells else None
        d.capacity_cells = self.cap_cells
        d.n_cells = self.counts.data_ptr() + 8
        d.stats = self.stats.data_ptr()
        d.vert_xyz = self.verts.data_ptr() if cap_verts else None
        d.tri_idx = self.faces.data_ptr() if cap_verts else None
        d.capacity_verts = self.cap_verts
        d.n_verts = self.counts.data_ptr() + 16

    def stats_dict(self):
        v = self.stats.cpu().numpy()
        return {n: int(v[i]) for i, n in enumerate(STAT_FIELDS)}


def options(precision="fp32", tau_mode=GH_TAU_DIAGONAL, eps=None, sync=True, ray_block=0, mlp_tiles=0,
            method="hop") -> Options:
    o = Options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.tau_mode = int(tau_mode)
    o.eps = -1.0 if eps is None else float(eps)
    o.sync = 1 if sync else 0
    o.ray_block = int(ray_block)
    o.mlp_tiles = int(mlp_tiles)
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    return o


def polygonize_into(sdb: Sdb, N, bufs: Buffers, lo=-1.0, hi=1.0, precision="fp32", tau_mode=GH_TAU_DIAGONAL,
                    eps=None, sync=True, stream=None, ray_block=0, mlp_tiles=0, method="hop") -> int:
    """Runs gh_polygonize into preallocated buffers; returns the status code
    (GH_ERR_CAPACITY is returned, not raised)."""
    g = _grid(N, lo, hi)
    o = options(precision, tau_mode, eps, sync, ray_block, mlp_tiles, method)
    rc = lib().gh_polygonize(ctypes.byref(g), sdb.handle, ctypes.byref(o), ctypes.byref(bufs.desc),
                             _stream_ptr(stream))
    if rc not in (GH_OK, GH_ERR_CAPACITY):
        check(rc)
    return rc


def polygonize(sdb: Sdb, N, lo=-1.0, hi=1.0, precision="fp32", tau_mode=GH_TAU_DIAGONAL, keys=False, cells=False,
               eps=None, stream=None, method="hop", indexed=False) -> Mesh:
    """gh_polygonize with buffers sized (and re-sized) automatically; returns
    device tensors trimmed to the produced counts.  indexed=True also returns
    the on-device indexed mesh (Mesh.verts, Mesh.faces)."""
    keys = bool(keys) or bool(indexed)
    key = (int(N), keys, bool(cells), bool(indexed))
    cap = sdb._cap.get(key, 4 * int(N) * int(N) + 4096)
    for _ in range(3):
        capv = cap // 2 + 4096 if indexed else 0
        bufs = Buffers(cap, keys=keys, cap_cells=cap if cells else 0, cap_verts=capv)
        rc = polygonize_into(sdb, N, bufs, lo, hi, precision, tau_mode, eps, True, stream, method=method)
        counts = bufs.counts.cpu().numpy()
        if rc == GH_OK:
            sdb._cap[key] = cap
            T, C, V = int(counts[0]), int(counts[1]), int(counts[2])
            return Mesh(bufs.tri_xyz[:T], bufs.tri_keys[:T] if keys else None,
                        bufs.cell_ids[:C] if cells else None, bufs.cell_cases[:C] if cells else None,
                        bufs.stats_dict(), bufs.verts[:V] if indexed else None,
                        bufs.faces[:T] if indexed else None)
        cap = int(max(counts[0], counts[1], 2 * counts[2]) * 1.1) + 4096
    raise GhError(GH_ERR_CAPACITY, "output buffers kept overflowing")


def polygonize_cont_into(sdb: Sdb, N, seeds, bufs: Buffers, lo=-1.0, hi=1.0, sync=True, stream=None) -> int:
    """gh_polygonize_cont (continuation from seed points, analytic SDBs) into
    preallocated buffers; returns the status (GH_ERR_CAPACITY returned)."""
    sp = np.ascontiguousarray(seeds, np.float32).reshape(-1, 3)
    g = _grid(N, lo, hi)
    o = options("fp32", GH_TAU_DIAGONAL, None, sync)
    rc = lib().gh_polygonize_cont(ctypes.byref(g), sdb.handle, sp.ctypes.data, sp.shape[0], ctypes.byref(o),
                                  ctypes.byref(bufs.desc), _stream_ptr(stream))
    if rc not in (GH_OK, GH_ERR_CAPACITY):
        check(rc)
    return rc


def polygonize_cont(sdb: Sdb, N, seeds, lo=-1.0, hi=1.0, keys=False, cells=False, stream=None) -> Mesh:
    """Continuation with buffers sized automatically (see polygonize)."""
    cap = 4 * int(N) * int(N) + 4096
    for _ in range(3):
        bufs = Buffers(cap, keys=keys, cap_cells=cap if cells else 0)
        rc = polygonize_cont_into(sdb, N, seeds, bufs, lo, hi, True, stream)
        counts = bufs.counts.cpu().numpy()
        if rc == GH_OK:
            T, C = int(counts[0]), int(counts[1])
            return Mesh(bufs.tri_xyz[:T], bufs.tri_keys[:T] if keys else None,
                        bufs.cell_ids[:C] if cells else None, bufs.cell_cases[:C] if cells else None,
                        bufs.stats_dict())
        cap = int(max(counts[0], counts[1]) * 1.1) + 4096
    raise GhError(GH_ERR_CAPACITY, "output buffers kept overflowing")


class Batch:
    """A batch of polygonizations bound to caller-owned buffers (one Buffers
    per item): run() executes gh_polygonize_batch; capture() builds a CUDA
    graph of the same launches that replay() re-runs."""

    def __init__(self, sdbs, Ns, caps, lo=-1.0, hi=1.0, precision="fp32", keys=False, eps=None, ray_block=0,
                 mlp_tiles=0, indexed=False, cells=False):
        self.sdbs = list(sdbs)
        self.Ns = [int(n) for n in Ns]
        self.B = len(self.sdbs)
        self.bufs = [Buffers(c, keys=keys, cap_cells=c if cells else 0, cap_verts=(c // 2 + 4096) if indexed else 0)
                     for c in caps]
        self.grids = (Grid * self.B)(*[_grid(n, lo, hi) for n in self.Ns])
        self.handles = (ctypes.c_void_p * self.B)(*[s_.handle for s_ in self.sdbs])
        self.meshes = (MeshDesc * self.B)(*[b.desc for b in self.bufs])
        self.opts = options(precision, GH_TAU_DIAGONAL, eps, True, ray_block, mlp_tiles)
        self.graph = None

    def run(self, sync=True, stream=None) -> int:
        self.opts.sync = 1 if sync else 0
        rc = lib().gh_polygonize_batch(self.B, self.grids, self.handles, ctypes.byref(self.opts), self.meshes,
                                       _stream_ptr(stream), None)
        if rc not in (GH_OK, GH_ERR_CAPACITY):
            check(rc)
        return rc

    def capture(self, stream=None):
        g = ctypes.c_void_p()
        check(lib().gh_polygonize_batch(self.B, self.grids, self.handles, ctypes.byref(self.opts), self.meshes,
                                        _stream_ptr(stream), ctypes.byref(g)))
        self.graph = g
        return g

    def replay(self, stream=None):
        check(lib().gh_batch_graph_launch(self.graph, _stream_ptr(stream)))

    def close(self):
        if self.graph is not None and _lib is not None:
            _lib.gh_batch_graph_free(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counts(self):
        import torch

        # triangles (or surface cells) needed, or twice the mesh vertices when those overflowed
        return torch.stack([torch.maximum(torch.maximum(b.counts[0], b.counts[1]), 2 * b.counts[2])
                            for b in self.bufs]).cpu().numpy()

    def mesh(self, b) -> "Mesh":
        bb = self.bufs[b]
        T, C, V = [int(x) for x in bb.counts.cpu().numpy()]
        ind = bb.verts is not None
        cl = bb.cell_ids is not None
        return Mesh(bb.tri_xyz[:T], bb.tri_keys[:T] if bb.tri_keys is not None else None,
                    bb.cell_ids[:C] if cl else None, bb.cell_cases[:C] if cl else None,
                    bb.stats_dict(), bb.verts[:V] if ind else None, bb.faces[:T] if ind else None)


def polygonize_batch(sdbs, Ns, lo=-1.0, hi=1.0, precision="fp32", keys=False, eps=None, ray_block=0, mlp_tiles=0,
                     indexed=False, cells=False):
    """gh_polygonize_batch with per-item buffers sized automatically; returns
    the Batch (its meshes via .mesh(b))."""
    caps = [4 * n * n + 4096 for n in Ns]
    for _ in range(3):
        bt = Batch(sdbs, Ns, caps, lo, hi, precision, keys, eps, ray_block, mlp_tiles, indexed, cells)
        rc = bt.run(sync=True)
        if rc == GH_OK:
            return bt
        need = bt.counts()
        caps = [int(max(c, n) * 1.1) + 4096 for c, n in zip(caps, need)]
    raise GhError(GH_ERR_CAPACITY, "batch buffers kept overflowing")


NOALLOC_MAX_N = 256
ADJOINT_CHUNK = 131072  # GH_ADJOINT_CHUNK: vertices per chunk of gh_backward


def csg_prims_device(prims, device=None):
    """The gh_csg_prim records of a scene as a device uint8 tensor (the input
    of polygonize_csg_noalloc, which copies nothing itself)."""
    import torch

    rec = np.frombuffer(csg_blob(prims)[16:], np.uint8).copy()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    return torch.from_numpy(rec).to(dev)


def polygonize_csg_noalloc(prims_dev, n_prim, N, bufs: Buffers, lo=-1.0, hi=1.0, tau_mode=GH_TAU_DIAGONAL,
                           stream=None) -> int:
    """gh_polygonize_csg_noalloc: the analytic pipeline on the library's
    static scratch (for callers that cannot allocate device memory); prims_dev
    from csg_prims_device.  Returns GH_OK or GH_ERR_CAPACITY, raises otherwise."""
    g = _grid(N, lo, hi)
    rc = lib().gh_polygonize_csg_noalloc(ctypes.byref(g), prims_dev.data_ptr(), int(n_prim), int(tau_mode),
                                         ctypes.byref(bufs.desc), _stream_ptr(stream))
    if rc not in (GH_OK, GH_ERR_CAPACITY):
        check(rc)
    return rc


def backward(sdb: Sdb, verts, dl_dv, stream=None):
    """gh_backward: dL/dtheta of a loss on mesh vertices through the implicit
    rule dv/dtheta = -grad f (df/dtheta)/|grad f|^2.  Neural SDB: packed like
    the MLP parameters.  Analytic SDB: [n_prim, 20] laid out like the
    primitive records (centre gradient in columns 2..4, size-parameter
    gradient in 5..7)."""
    import torch

    v = verts.detach().contiguous().to(torch.float32)
    g = dl_dv.detach().contiguous().to(torch.float32)
    n = sdb.params.size if isinstance(sdb, MlpSdb) else sdb.prims.shape[0] * 20
    out = torch.empty(n, dtype=torch.float32, device=v.device)
    check(lib().gh_backward(sdb.handle, v.data_ptr(), g.data_ptr(), v.shape[0], out.data_ptr(),
                            _stream_ptr(stream)))
    return out if isinstance(sdb, MlpSdb) else out.reshape(-1, 20)


def eval_points(sdb: Sdb, pts, precision="fp32", stream=None):
    """f at points [n,3] (a torch CUDA float32 tensor) -> [n] float32."""
    import torch

    p = pts.contiguous().to(torch.float32)
    out = torch.empty(p.shape[0], dtype=torch.float32, device=p.device)
    check(lib().gh_eval(sdb.handle, p.data_ptr(), p.shape[0], out.data_ptr(), PRECISIONS[precision],
                        _stream_ptr(stream)))
    return out


def set_wait_limit_ns(ns: int):
    """gh_set_wait_limit_ns: limit of the neural engines' bounded waits (2e9 =
    2 s, the default; 0 = every wait on the engines' own work runs out at once)."""
    check(lib().gh_set_wait_limit_ns(int(ns)))


def release_cache():
    """Frees the scratch the library keeps from destroyed SDBs (gh_release_cache)."""
    check(lib().gh_release_cache())


def set_profiling(enable: bool):
    check(lib().gh_set_profiling(1 if enable else 0))


def last_profile():
    """(launches, {phase: ms}) of the last gh_polygonize on this thread."""
    p = Profile()
    check(lib().gh_last_profile(ctypes.byref(p)))
    return int(p.launches), ({PHASES[i]: float(p.ms[i]) for i in range(p.n_phases)} if p.n_phases else {})


def version() -> str:
    return lib().gh_version().decode()


def column_order(N, c):
    """gh_column_order: the column the c-th claim of the hoppers' queue takes."""
    return int(lib().gh_column_order(int(N), int(c)))
