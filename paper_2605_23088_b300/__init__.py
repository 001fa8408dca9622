"""B300-native IPC Newton hot path (YASPS, arxiv 2605.23088) -- Python binding.

A thin ctypes binding over the C ABI of ``libyasps.so`` (declared in
``include/yasps.h``).  It only marshals arguments: every step of the path
(element and barrier derivatives, projection, assembly, PCG, broadphase, CCD,
line search) runs in the library's CUDA kernels.  PyTorch provides the device
memory (the library's workspaces come from torch's caching allocator through
the allocator callbacks) and the CUDA stream.  There is no CPU fallback: if
the library or a CUDA device is missing, the calls raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libyasps.so")

YASPS_OK = 0
STATUS = {0: "OK", -1: "E_INVAL", -2: "E_NOMEM", -3: "E_CUDA", -4: "E_CAPACITY", -5: "E_NOCONV",
          -6: "E_LINESEARCH", -7: "E_TIMEOUT", -8: "E_NAN"}
TERM_INERTIA, TERM_TET, TERM_MEMBRANE, TERM_BEND, TERM_ABD, TERM_BARRIER, TERM_ALL = 1, 2, 4, 8, 16, 32, 63

# every symbol include/yasps.h declares
EXPORTS = [
    "yasps_default_params", "yasps_build_system", "yasps_build_error", "yasps_destroy", "yasps_last_error",
    "yasps_set_params", "yasps_get_sizes", "yasps_initial_state", "yasps_vertex_positions", "yasps_xtilde",
    "yasps_detect_pairs", "yasps_export_pairs", "yasps_energy", "yasps_eval_local", "yasps_assemble",
    "yasps_export_bsr", "yasps_export_gradient", "yasps_spmv", "yasps_pcg_solve", "yasps_ccd_bound", "yasps_step",
    "yasps_set_fixed_positions", "yasps_get_fixed_positions", "yasps_set_tet_young", "yasps_adjoint_step", "yasps_scene_stats", "yasps_autotune_pcg", "yasps_set_pcg_variant", "yasps_kernel_launches", "yasps_profile_enable",
    "yasps_profile_get", "yasps_pcg_phase_ms", "yasps_pcg_block_busy", "yasps_pcg_solve_static", "yasps_newton_trace",
    "yasps_newton_trace_enable", "yasps_get_kappa_state", "yasps_set_kappa_state", "yasps_set_wait_limit",
    "yasps_probe_fma_tflops", "yasps_spmv_format", "yasps_project_batch",
]
SPMV_UPPER_BSR, SPMV_FULL_BSR, SPMV_FULL_BCOO, SPMV_UPPER_BCOO = range(4)
SPMV_FORMATS = ["upper_bsr", "full_bsr", "full_bcoo", "upper_bcoo"]
STAGE_SPMV, STAGE_TET, STAGE_BARRIER, STAGE_PCG, STAGE_DETECT, STAGE_EVAL, STAGE_CCD, STAGE_LS, STAGE_PCG_KERNEL = range(9)
STAGE_NAMES = ["spmv", "tet", "barrier", "pcg", "detect", "eval", "ccd", "line_search", "pcg_kernel"]
PCG_VARIANTS = 5  # YASPS_PCG_VARIANTS
PCG_PHASES = ["own_nodes", "upper_blocks", "wait_dHd", "update", "wait_rz", "hd_busy_mean", "hd_busy_max", "wait_dn"]


class YaspsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("dt", ctypes.c_double), ("dhat", ctypes.c_double),
                ("kappa", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("newton_tol", ctypes.c_double),
                ("pcg_rel_tol", ctypes.c_double), ("pcg_max_iter", ctypes.c_int), ("newton_max_iter", ctypes.c_int),
                ("ls_max_iter", ctypes.c_int), ("barrier_form", ctypes.c_int), ("ccd_gap", ctypes.c_double),
                ("ccd_max_iter", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("pcg_warm_start", ctypes.c_int),
                ("kappa_adaptive", ctypes.c_int), ("kappa_min", ctypes.c_double), ("kappa_max", ctypes.c_double),
                ("kappa_dmin", ctypes.c_double), ("ls_armijo", ctypes.c_double)]


_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


class SceneDesc(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int), ("rest_pos", _PD), ("vert_body", _PI),
                ("n_fixed", ctypes.c_int), ("fixed_verts", _PI), ("fixed_vel", _PD),
                ("n_tets", ctypes.c_int), ("tet2v", _PI), ("tet_E", _PD), ("tet_nu", _PD), ("tet_rho", _PD),
                ("n_tris", ctypes.c_int), ("tri2v", _PI), ("tri_E", _PD), ("tri_nu", _PD), ("tri_thick", _PD),
                ("tri_rho", _PD),
                ("n_hinges", ctypes.c_int), ("hinge2v", _PI), ("hinge_kb", _PD),
                ("n_bodies", ctypes.c_int), ("body_mass", _PD), ("body_vol", _PD), ("body_kappa", _PD),
                ("n_surf_tris", ctypes.c_int), ("surf_tri2v", _PI), ("n_surf_edges", ctypes.c_int),
                ("surf_edge2v", _PI), ("n_surf_verts", ctypes.c_int), ("surf_verts", _PI),
                ("n_planes", ctypes.c_int), ("planes", _PD), ("n_scenes", ctypes.c_int), ("vert_scene", _PI),
                ("cloth_model", ctypes.c_int), ("tri_shear", _PD), ("n_embedded", ctypes.c_int),
                ("embed_verts", _PI), ("embed_cage", _PI), ("embed_w", _PD)]


class StepStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("pcg_iters_total", ctypes.c_int), ("n_pt", ctypes.c_int),
                ("n_ee", ctypes.c_int), ("n_pg", ctypes.c_int), ("status", ctypes.c_int),
                ("alpha_last", ctypes.c_double), ("p_inf", ctypes.c_double), ("t_eval_ms", ctypes.c_double),
                ("t_pcg_ms", ctypes.c_double), ("t_ccd_ms", ctypes.c_double), ("t_ls_ms", ctypes.c_double),
                ("n_cand_pt", ctypes.c_int), ("n_cand_ee", ctypes.c_int), ("kappa", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NewtonRecord(ctypes.Structure):
    _fields_ = [("pcg_iters", ctypes.c_int), ("ls_halvings", ctypes.c_int), ("n_pt", ctypes.c_int),
                ("n_ee", ctypes.c_int), ("n_pg", ctypes.c_int), ("n_cand_pt", ctypes.c_int),
                ("n_cand_ee", ctypes.c_int), ("pinf_node", ctypes.c_int), ("p_inf", ctypes.c_double),
                ("pcg_rel_res", ctypes.c_double), ("alpha_ccd", ctypes.c_double), ("alpha", ctypes.c_double),
                ("E0", ctypes.c_double), ("E1", ctypes.c_double), ("s_min", ctypes.c_double),
                ("g_dot_p", ctypes.c_double), ("p_at_max", ctypes.c_double * 3)]


class StageStats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_longlong), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Allocator(ctypes.Structure):
    _ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    _FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC), ("free", _FREE)]


_lib = None


def lib():
    """Load libyasps.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2605_23088_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        L.yasps_build_error.restype = ctypes.c_char_p
        L.yasps_last_error.restype = ctypes.c_char_p
        L.yasps_kernel_launches.restype = ctypes.c_longlong
        L.yasps_build_system.argtypes = [ctypes.POINTER(SceneDesc), ctypes.POINTER(Params),
                                         ctypes.POINTER(Allocator), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def default_params(**kw):
    p = Params()
    lib().yasps_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "gravity":
            p.gravity[:] = list(v)
        else:
            setattr(p, k, v)
    return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def spmv_format(fmt, n_nodes, row, col, vals, diag, x, y, flag, stream=None):
    """y = (D + A_off) x in one of the four layouts of the SpMV study
    (yasps_spmv_format); every argument a contiguous CUDA tensor (row, col,
    flag int32; vals [nnzb,3,3], diag [n,3,3], x, y [n,3] all float64 or all
    float32).  Asynchronous on the stream."""
    import torch

    prec = 0 if x.dtype == torch.float64 else 1
    s = stream if stream is not None else torch.cuda.current_stream()
    nnzb = int(row.numel())
    null = ctypes.c_void_p(0)
    rc = lib().yasps_spmv_format(ctypes.c_int(fmt), ctypes.c_int(prec), ctypes.c_int(n_nodes), ctypes.c_int(nnzb),
                                 _ptr(row) if nnzb else null, _ptr(col) if nnzb else null,
                                 _ptr(vals) if nnzb else null, _ptr(diag), _ptr(x), _ptr(y), _ptr(flag),
                                 ctypes.c_void_p(s.cuda_stream))
    if rc != YASPS_OK:
        raise YaspsError(rc, "yasps_spmv_format failed")


def project_batch(H, out=None, stream=None):
    """PSD projection of a batch of symmetric matrices H (CUDA tensor [count, n, n],
    float64 or float32, n in 3, 6, 9, 12, 15, 24) by the library's warp Jacobi."""
    import torch

    if out is None:
        out = torch.empty_like(H)
    count, n = int(H.shape[0]), int(H.shape[1])
    prec = 0 if H.dtype == torch.float64 else 1
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().yasps_project_batch(ctypes.c_int(n), ctypes.c_int(count), ctypes.c_int(prec), _ptr(H), _ptr(out),
                                   ctypes.c_void_p(s.cuda_stream))
    if rc != YASPS_OK:
        raise YaspsError(rc, "yasps_project_batch failed")
    return out


def probe_fma_tflops(precision):
    """Measured FMA throughput of the current GPU's FP64 (0) or FP32 (1) pipe, TFLOP/s."""
    t = ctypes.c_double()
    rc = lib().yasps_probe_fma_tflops(ctypes.c_int(precision), ctypes.byref(t))
    if rc != YASPS_OK:
        raise YaspsError(rc, "FMA probe failed")
    return t.value


def pcg_solve_static(n_nodes, row, col, vals, diag, rhs, rel_tol=1e-4, max_iter=0, stream=None, out=None):
    """Block-Jacobi PCG that allocates no device memory (yasps_pcg_solve_static).

    For callers that may not allocate at solve time: every argument is a
    contiguous CUDA tensor the caller owns (row/col int32 [nnzb], vals float64
    [nnzb,3,3], diag float64 [n_nodes,3,3], rhs float64 [n_nodes,3]); the
    temporaries live in a fixed device array inside the library (at most 65536
    nodes).  ``out`` (float64 [n_nodes,3], not aliasing rhs) receives p; without
    it a new tensor is made here (which allocates, on the caller's side).
    Returns (p, iters, rel_res).
    """
    import torch

    nnzb = int(row.numel())
    want = [("row", row, torch.int32, (nnzb,)), ("col", col, torch.int32, (nnzb,)),
            ("vals", vals, torch.float64, (nnzb, 3, 3)), ("diag", diag, torch.float64, (n_nodes, 3, 3)),
            ("rhs", rhs, torch.float64, (n_nodes, 3))]
    if out is not None:
        want.append(("out", out, torch.float64, (n_nodes, 3)))
    for name, t, dt, shape in want:
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"pcg_solve_static: {name} must be a contiguous CUDA {dt} tensor")
        if tuple(t.shape) != shape and not (t.numel() == 0 and 0 in shape):
            raise ValueError(f"pcg_solve_static: {name} has shape {tuple(t.shape)}, expected {shape}")
    p = torch.empty_like(rhs) if out is None else out
    it, rel = ctypes.c_int(), ctypes.c_double()
    err = ctypes.create_string_buffer(256)
    s = stream if stream is not None else torch.cuda.current_stream()
    null = ctypes.c_void_p(0)
    rc = lib().yasps_pcg_solve_static(ctypes.c_int(n_nodes), ctypes.c_int(nnzb), _ptr(row) if nnzb else null,
                                      _ptr(col) if nnzb else null, _ptr(vals) if nnzb else null, _ptr(diag),
                                      _ptr(rhs), _ptr(p), ctypes.c_double(rel_tol), ctypes.c_int(max_iter),
                                      ctypes.c_void_p(s.cuda_stream), ctypes.byref(it), ctypes.byref(rel), err,
                                      ctypes.c_int(len(err)))
    if rc != YASPS_OK:
        raise YaspsError(rc, err.value.decode())
    return p, it.value, rel.value


class System:
    """A scene held on the GPU by the library (one ``yasps_system``).

    ``scene`` is a dict from the ``scenes`` generators.  State tensors (x, v)
    are torch FP64 CUDA tensors of shape (n_nodes, 3).
    """

    def __init__(self, scene, use_torch_allocator=True, stream=None, **params):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2605_23088_b300 needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p = dict(dt=scene["dt"], dhat=scene["dhat"], kappa=scene["kappa"], gravity=list(scene["gravity"]),
                 newton_tol=scene["newton_tol"])
        p.update(params)
        self.params = default_params(**p)
        self._keep = []

        def arr(a, dtype):
            a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
            self._keep.append(a)
            return a.ctypes.data_as(_PD if dtype == np.float64 else _PI)

        s = scene
        d = SceneDesc()
        d.n_verts = len(s["rest_pos"]); d.rest_pos = arr(s["rest_pos"], np.float64); d.vert_body = arr(s["vert_body"], np.int32)
        d.n_fixed = len(s["fixed"]); d.fixed_verts = arr(s["fixed"], np.int32); d.fixed_vel = arr(s["fixed_vel"], np.float64)
        d.n_tets = len(s["tets"]); d.tet2v = arr(s["tets"], np.int32); d.tet_E = arr(s["tet_E"], np.float64)
        d.tet_nu = arr(s["tet_nu"], np.float64); d.tet_rho = arr(s["tet_rho"], np.float64)
        d.n_tris = len(s["tris"]); d.tri2v = arr(s["tris"], np.int32); d.tri_E = arr(s["tri_E"], np.float64)
        d.tri_nu = arr(s["tri_nu"], np.float64); d.tri_thick = arr(s["tri_thick"], np.float64)
        d.tri_rho = arr(s["tri_rho"], np.float64)
        d.n_hinges = len(s["hinges"]); d.hinge2v = arr(s["hinges"], np.int32); d.hinge_kb = arr(s["hinge_kb"], np.float64)
        d.n_bodies = len(s["body_mass"]); d.body_mass = arr(s["body_mass"], np.float64)
        d.body_vol = arr(s["body_vol"], np.float64); d.body_kappa = arr(s["body_kappa"], np.float64)
        d.n_surf_tris = len(s["surf_tris"]); d.surf_tri2v = arr(s["surf_tris"], np.int32)
        d.n_surf_edges = len(s["surf_edges"]); d.surf_edge2v = arr(s["surf_edges"], np.int32)
        d.n_surf_verts = len(s["surf_verts"]); d.surf_verts = arr(s["surf_verts"], np.int32)
        d.n_planes = len(s["planes"]); d.planes = arr(s["planes"], np.float64)
        if len(s.get("embed_verts", ())):
            d.n_embedded = len(s["embed_verts"]); d.embed_verts = arr(s["embed_verts"], np.int32)
            d.embed_cage = arr(s["embed_cage"], np.int32); d.embed_w = arr(s["embed_w"], np.float64)
        d.cloth_model = int(s.get("cloth_model", 0))
        if d.cloth_model:
            d.tri_shear = arr(s["tri_shear"], np.float64)
        if s.get("vert_scene") is not None and int(s.get("n_scenes", 1)) > 1:
            d.n_scenes = int(s["n_scenes"]); d.vert_scene = arr(s["vert_scene"], np.int32)
        self.n_scenes = max(1, int(d.n_scenes))
        self.scene = scene
        self._alloc = None
        if use_torch_allocator:
            dev = self.device.index

            def _a(ctx, nbytes, stream):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))

            def _f(ctx, ptr, stream):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (Allocator._ALLOC(_a), Allocator._FREE(_f))
            self._alloc = Allocator(None, self._cb[0], self._cb[1])
        h = ctypes.c_void_p()
        rc = lib().yasps_build_system(ctypes.byref(d), ctypes.byref(self.params),
                                      ctypes.byref(self._alloc) if self._alloc else None,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != YASPS_OK:
            raise YaspsError(rc, lib().yasps_build_error().decode())
        self.h = h
        nn, nf, nv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib().yasps_get_sizes(self.h, ctypes.byref(nn), ctypes.byref(nf), ctypes.byref(nv))
        self.n_nodes, self.n_free, self.n_verts = nn.value, nf.value, nv.value

    # ------------------------------------------------------------ plumbing
    def _check(self, rc):
        if rc != YASPS_OK:
            raise YaspsError(rc, lib().yasps_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().yasps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, *shape, dtype=None):
        return self.torch.zeros(*shape, dtype=dtype or self.torch.float64, device=self.device)

    # ------------------------------------------------------------ ABI calls
    def set_params(self, **kw):
        for k, v in kw.items():
            if k == "gravity":
                self.params.gravity[:] = list(v)
            else:
                setattr(self.params, k, v)
        self._check(lib().yasps_set_params(self.h, ctypes.byref(self.params)))

    def initial_state(self):
        x = self.zeros(self.n_nodes, 3)
        v = self.zeros(self.n_nodes, 3)
        vel0 = np.ascontiguousarray(self.scene["vel0"], dtype=np.float64)
        self._check(lib().yasps_initial_state(self.h, vel0.ctypes.data_as(_PD), _ptr(x), _ptr(v)))
        return x, v

    def vertex_positions(self, x):
        P = self.zeros(self.n_verts, 3)
        self._check(lib().yasps_vertex_positions(self.h, _ptr(x), _ptr(P)))
        return P

    def xtilde(self, x, v):
        out = self.zeros(self.n_nodes, 3)
        self._check(lib().yasps_xtilde(self.h, _ptr(x), _ptr(v), _ptr(out)))
        return out

    def detect_pairs(self, x):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().yasps_detect_pairs(self.h, _ptr(x), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def export_pairs(self, counts):
        pt = np.zeros((counts[0], 3), np.int32)
        ee = np.zeros((counts[1], 3), np.int32)
        pg = np.zeros((counts[2], 3), np.int32)
        self._check(lib().yasps_export_pairs(self.h, pt.ctypes.data_as(_PI), ee.ctypes.data_as(_PI),
                                             pg.ctypes.data_as(_PI)))
        return pt, ee, pg

    def pairs(self, x):
        return self.export_pairs(self.detect_pairs(x))

    def energy(self, x, xtil, terms=False):
        E = ctypes.c_double()
        t = np.zeros(6)
        self._check(lib().yasps_energy(self.h, _ptr(x), _ptr(xtil), ctypes.byref(E), t.ctypes.data_as(_PD)))
        return (E.value, t) if terms else E.value

    def eval_local(self, x, xtil, term_mask=TERM_ALL, project=True):
        self._check(lib().yasps_eval_local(self.h, _ptr(x), _ptr(xtil), ctypes.c_int(term_mask),
                                           ctypes.c_int(int(project))))

    def assemble(self):
        self._check(lib().yasps_assemble(self.h))

    def bsr_nnzb(self, which):
        """Number of upper blocks of the static (0) or dynamic (1) BSR part."""
        nnzb = ctypes.c_int()
        self._check(lib().yasps_export_bsr(self.h, ctypes.c_int(which), ctypes.byref(nnzb), None, None, None, None))
        return nnzb.value

    def export_bsr(self, which):
        nnzb = ctypes.c_int()
        self._check(lib().yasps_export_bsr(self.h, ctypes.c_int(which), ctypes.byref(nnzb), None, None, None, None))
        n = nnzb.value
        rowptr = np.zeros(self.n_nodes + 1, np.int32)
        col = np.zeros(max(n, 1), np.int32)
        vals = np.zeros((max(n, 1), 9))
        diag = np.zeros((self.n_nodes, 9))
        self._check(lib().yasps_export_bsr(self.h, ctypes.c_int(which), ctypes.byref(nnzb), rowptr.ctypes.data_as(_PI),
                                           col.ctypes.data_as(_PI), vals.ctypes.data_as(_PD),
                                           diag.ctypes.data_as(_PD) if which == 0 else None))
        return rowptr, col[:n].copy(), vals[:n].reshape(n, 3, 3).copy(), diag.reshape(-1, 3, 3)

    def export_gradient(self):
        g = self.zeros(self.n_nodes, 3)
        self._check(lib().yasps_export_gradient(self.h, _ptr(g)))
        return g

    def spmv(self, x):
        y = self.zeros(self.n_nodes, 3)
        self._check(lib().yasps_spmv(self.h, _ptr(x), _ptr(y)))
        return y

    def pcg_solve(self, rhs, rel_tol=1e-4):
        p = self.zeros(self.n_nodes, 3)
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._check(lib().yasps_pcg_solve(self.h, _ptr(rhs), _ptr(p), ctypes.c_double(rel_tol), ctypes.byref(it),
                                          ctypes.byref(rel)))
        return p, it.value, rel.value

    def ccd_bound(self, x, p):
        a = ctypes.c_double()
        self._check(lib().yasps_ccd_bound(self.h, _ptr(x), _ptr(p), ctypes.byref(a)))
        return a.value

    def step(self, x, v, raise_on_error=True):
        """One implicit time step, x and v updated in place; returns the stats dict."""
        st = StepStats()
        rc = lib().yasps_step(self.h, _ptr(x), _ptr(v), ctypes.byref(st))
        if raise_on_error:
            self._check(rc)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def newton_trace(self):
        """Per-Newton-iteration records of the last step (list of dicts, yasps_newton_trace)."""
        n = ctypes.c_int()
        self._check(lib().yasps_newton_trace(self.h, ctypes.c_int(0), None, ctypes.byref(n)))
        recs = (NewtonRecord * max(n.value, 1))()
        self._check(lib().yasps_newton_trace(self.h, ctypes.c_int(n.value), recs, ctypes.byref(n)))
        out = []
        for r in recs[:n.value]:
            d = {k: getattr(r, k) for k, _ in NewtonRecord._fields_}
            d["p_at_max"] = list(r.p_at_max)
            out.append(d)
        return out

    def newton_trace_enable(self, on=True):
        """Also record the smallest pair distance of every Newton iteration."""
        self._check(lib().yasps_newton_trace_enable(self.h, ctypes.c_int(int(on))))

    def kappa_state(self):
        """(kappa, initialised, smallest pair distance at the previous step's start,
        lower bound, upper bound) of the adaptive barrier stiffness."""
        k, i, d, lo, hi = ctypes.c_double(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(lib().yasps_get_kappa_state(self.h, ctypes.byref(k), ctypes.byref(i), ctypes.byref(d),
                                                ctypes.byref(lo), ctypes.byref(hi)))
        return k.value, bool(i.value), d.value, lo.value, hi.value

    def set_kappa_state(self, kappa, initialised, dmin_prev):
        self._check(lib().yasps_set_kappa_state(self.h, ctypes.c_double(kappa), ctypes.c_int(int(initialised)),
                                                ctypes.c_double(dmin_prev)))

    def set_fixed_positions(self, P):
        P = np.ascontiguousarray(P, dtype=np.float64)
        self._check(lib().yasps_set_fixed_positions(self.h, P.ctypes.data_as(_PD)))

    def get_fixed_positions(self):
        P = np.zeros((self.n_verts, 3))
        self._check(lib().yasps_get_fixed_positions(self.h, P.ctypes.data_as(_PD)))
        return P

    def autotune_pcg(self, iters=30):
        """Time each PCG launch configuration on the current assembly and keep the
        fastest; returns (variant, microseconds per iteration of each)."""
        v = ctypes.c_int()
        us = np.zeros(PCG_VARIANTS)
        self._check(lib().yasps_autotune_pcg(self.h, ctypes.c_int(iters), ctypes.byref(v), us.ctypes.data_as(_PD)))
        return v.value, us

    def set_wait_limit(self, polls, unmet_next=False):
        """Polls a PCG-kernel wait may spend before the solve gives up with E_TIMEOUT
        (0: default); unmet_next makes the next launch's barriers wait for an
        arrival that never comes (testing the timeout path)."""
        self._check(lib().yasps_set_wait_limit(self.h, ctypes.c_longlong(int(polls)), ctypes.c_int(int(unmet_next))))

    def set_pcg_variant(self, variant):
        self._check(lib().yasps_set_pcg_variant(self.h, ctypes.c_int(variant)))

    def scene_stats(self):
        """Per-scene (Newton iterations, PCG iterations, status) of the last step (batches)."""
        n = self.n_scenes
        a, b, c = (np.zeros(n, np.int32) for _ in range(3))
        self._check(lib().yasps_scene_stats(self.h, a.ctypes.data_as(_PI), b.ctypes.data_as(_PI), c.ctypes.data_as(_PI)))
        return a, b, c

    def set_tet_young(self, E):
        """Per-tet Young's moduli (CUDA float64 tensor [n_tets]); Poisson ratios kept."""
        E = E.detach().to(device=self.device, dtype=self.torch.float64).contiguous()
        self._check(lib().yasps_set_tet_young(self.h, _ptr(E)))

    def adjoint_step(self, x_t, v_t, x_next, xbar, vbar, Ebar, tol=1e-10):
        """One reverse step (yasps_adjoint_step): returns (dL/dx_t, dL/dv_t, PCG iterations,
        relative residual) and adds this step's dL/dE into Ebar in place."""
        xp = self.zeros(self.n_nodes, 3)
        vp = self.zeros(self.n_nodes, 3)
        it, rel = ctypes.c_int(), ctypes.c_double()
        self._check(lib().yasps_adjoint_step(self.h, _ptr(x_t), _ptr(v_t), _ptr(x_next), _ptr(xbar), _ptr(vbar),
                                             _ptr(xp), _ptr(vp), _ptr(Ebar), ctypes.c_double(tol),
                                             ctypes.byref(it), ctypes.byref(rel)))
        return xp, vp, it.value, rel.value

    def kernel_launches(self):
        return lib().yasps_kernel_launches(self.h)

    def profile_enable(self, on=True):
        self._check(lib().yasps_profile_enable(self.h, ctypes.c_int(int(on))))

    def profile_get(self, stage):
        st = StageStats()
        self._check(lib().yasps_profile_get(self.h, ctypes.c_int(stage), ctypes.byref(st)))
        return {"count": st.count, "ms": st.ms, "bytes": st.bytes}

    def pcg_phase_ms(self):
        """Per-phase time of the PCG kernel while profiling (ms): own nodes' direction
        and diagonal product, upper blocks, wait + d^T H d, update, wait + r^T z."""
        out = np.zeros(8)
        self._check(lib().yasps_pcg_phase_ms(self.h, out.ctypes.data_as(_PD)))
        return dict(zip(PCG_PHASES, out.tolist()))

    def pcg_block_busy(self):
        """Per-block own-node + upper-block time of the PCG kernel (us per
        iteration) and the SM of each block, over the launches profiled since
        profile_enable(True)."""
        n = ctypes.c_int()
        self._check(lib().yasps_pcg_block_busy(self.h, 0, ctypes.byref(n), None, None))
        us = np.zeros(max(n.value, 1))
        sm = np.zeros(max(n.value, 1), np.int32)
        self._check(lib().yasps_pcg_block_busy(self.h, n.value, ctypes.byref(n), us.ctypes.data_as(_PD),
                                               sm.ctypes.data_as(_PI)))
        return us[:n.value], sm[:n.value]
