"""FP64 CPU oracle of the IPC Newton hot path -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
use this package.  The library (``paper_2605_23088_b300``) never imports it and
shares no code with it: the oracle is ``oracle.c`` (plain C, FP64,
``-ffp-contract=off``), loaded through ctypes by this thin wrapper.

Function-level parity status (each item is pinned by a ``-m "not gpu"`` test
against something other than the oracle itself, see tests/test_oracle_pins.py):
  Jacobi EVD / PSD projection   pinned (numpy eigh, nearest-PSD property)
  SNH (Eq. snh)                 pinned (rest-stability, FD, rotation invariance,
                                        closed-form F=I Hessian)
  StVK membrane, bending        pinned (FD, rigid-motion invariance, closed form
                                        of the flat hinge); constants are textbook,
                                        not the paper's (parity unpinned w.r.t. paper)
  ABD orthogonality             pinned (zero + zero gradient at rotations, FD)
  distances + classification    pinned (dense brute-force sampling, closed forms)
  barrier                       pinned (closed form, FD, C2 at dhat)
  pairs                         pinned (O(n^2) enumeration vs grid)
  BSR assembly                  pinned (dense assembly, dense FD Hessian)
  PCG                           pinned (numpy dense solve)
  ACCD                          pinned (no-crossing invariant, exact TOI cases)
  time step                     pinned (free-fall closed form, energy decrease,
                                        no interpenetration); post-contact
                                        trajectories: parity unpinned
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

D = ctypes.POINTER(ctypes.c_double)
I = ctypes.POINTER(ctypes.c_int)


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, FP64, no FP contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
    subprocess.check_call(cmd)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.or_create.restype = ctypes.c_void_p
        _lib.or_energy.restype = ctypes.c_double
        _lib.or_accd.restype = ctypes.c_double
        _lib.or_pg_ccd.restype = ctypes.c_double
        _lib.or_ccd_bound.restype = ctypes.c_double
        _lib.or_get_kappa.restype = ctypes.c_double
    return _lib


def _dp(a):
    return a.ctypes.data_as(D)


def _ip(a):
    return a.ctypes.data_as(I)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# ---------------------------------------------------------------- elements
def eig_sym(A):
    A = _f64(A)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().or_eig_sym(ctypes.c_int(n), _dp(A), _dp(w), _dp(V))
    return w, V


def project_psd(A):
    A = _f64(A)
    n = A.shape[0]
    out = np.zeros((n, n))
    lib().or_project_psd(ctypes.c_int(n), _dp(A), _dp(out))
    return out


def lame(E, nu):
    mu, lam = ctypes.c_double(), ctypes.c_double()
    lib().or_lame(ctypes.c_double(E), ctypes.c_double(nu), ctypes.byref(mu), ctypes.byref(lam))
    return mu.value, lam.value


def lame_plane_stress(E, nu):
    mu, lam = ctypes.c_double(), ctypes.c_double()
    lib().or_lame_ps(ctypes.c_double(E), ctypes.c_double(nu), ctypes.byref(mu), ctypes.byref(lam))
    return mu.value, lam.value


def snh_Fspace(F, mu, lam):
    F = _f64(F).ravel()
    psi = ctypes.c_double()
    P = np.zeros(9)
    H = np.zeros(81)
    lib().or_snh_Fspace(_dp(F), ctypes.c_double(mu), ctypes.c_double(lam), ctypes.byref(psi), _dp(P), _dp(H))
    return psi.value, P, H.reshape(9, 9)


def _local(fn, n, x, X, *scal, project=True):
    x = _f64(x).ravel()
    X = _f64(X).ravel()
    E = ctypes.c_double()
    g = np.zeros(n)
    H = np.zeros(n * n)
    args = [ctypes.c_double(s) for s in scal]
    rc = fn(_dp(x), _dp(X), *args, ctypes.c_int(int(project)), ctypes.byref(E), _dp(g), _dp(H))
    if rc != 0:
        raise ValueError("degenerate rest element")
    return E.value, g, H.reshape(n, n)


def snh_local(x, X, mu, lam, project=True):
    return _local(lib().or_snh_local, 12, x, X, mu, lam, project=project)


def stvk_local(x, X, mu, lam, thick, project=True):
    return _local(lib().or_stvk_local, 9, x, X, mu, lam, thick, project=project)


def bend_local(x, X, kb, project=True):
    return _local(lib().or_bend_local, 12, x, X, kb, project=project)


def hinge_rest(X):
    X = _f64(X).ravel()
    th, w = ctypes.c_double(), ctypes.c_double()
    lib().or_hinge_rest(_dp(X), ctypes.byref(th), ctypes.byref(w))
    return th.value, w.value


def abd_ortho_local(A_cols, kv, project=True):
    A = _f64(A_cols).ravel()
    E = ctypes.c_double()
    g = np.zeros(9)
    H = np.zeros(81)
    lib().or_abd_ortho_local(_dp(A), ctypes.c_double(kv), ctypes.c_int(int(project)), ctypes.byref(E), _dp(g), _dp(H))
    return E.value, g, H.reshape(9, 9)


def barrier_scalar(s, shat, form=0):
    b, db, d2b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_barrier_scalar(ctypes.c_double(s), ctypes.c_double(shat), ctypes.c_int(form),
                            ctypes.byref(b), ctypes.byref(db), ctypes.byref(d2b))
    return b.value, db.value, d2b.value


def pt_classify(p, a, b, c):
    s = ctypes.c_double()
    st = lib().or_pt_classify(_dp(_f64(p)), _dp(_f64(a)), _dp(_f64(b)), _dp(_f64(c)), ctypes.byref(s))
    return st, s.value


def ee_classify(a0, a1, b0, b1):
    s = ctypes.c_double()
    st = lib().or_ee_classify(_dp(_f64(a0)), _dp(_f64(a1)), _dp(_f64(b0)), _dp(_f64(b1)), ctypes.byref(s))
    return st, s.value


def bw_local(x, X, kst, ksh, thick, project=True):
    """Baraff-Witkin stretch + shear membrane triangle: (energy, gradient 9, Hessian 9x9)."""
    return _local(lib().or_bw_local, 9, x, X, kst, ksh, thick, project=project)


def pair_local(kind, xloc, plane=None, kappa=1.0, shat=1e-6, form=0, project=True):
    """kind 0 = PT, 1 = EE, 2 = PG; returns (E, g, H, subtype) in position space."""
    xl = _f64(xloc).ravel()
    n = 3 if kind == 2 else 12
    pl = _f64(plane if plane is not None else np.zeros(4))
    E = ctypes.c_double()
    g = np.zeros(n)
    H = np.zeros(n * n)
    st = ctypes.c_int()
    lib().or_pair_local(ctypes.c_int(kind), _dp(xl), _dp(pl), ctypes.c_double(kappa), ctypes.c_double(shat),
                        ctypes.c_int(form), ctypes.c_int(int(project)), ctypes.byref(E), _dp(g), _dp(H), ctypes.byref(st))
    return E.value, g, H.reshape(n, n), st.value


def accd(kind, x, dx, gap_s=0.1, tmax=1.0, max_iter=100000):
    it = ctypes.c_int()
    t = lib().or_accd(ctypes.c_int(kind), _dp(_f64(x).ravel()), _dp(_f64(dx).ravel()), ctypes.c_double(gap_s),
                      ctypes.c_double(tmax), ctypes.c_int(max_iter), ctypes.byref(it))
    return t, it.value


def pg_ccd(p, dp, plane, gap_s=0.1, tmax=1.0):
    return lib().or_pg_ccd(_dp(_f64(p)), _dp(_f64(dp)), _dp(_f64(plane)), ctypes.c_double(gap_s), ctypes.c_double(tmax))


# ---------------------------------------------------------------- system
DEFAULT_PARAMS = dict(pcg_tol=1e-4, pcg_max=0, newton_max=100, ls_max=30, barrier_form=0, gap_s=0.1,
                      ccd_max_iter=100000)


class OracleSystem:
    """A scene (from the ``scenes`` generators) held by the C oracle."""

    def __init__(self, scene, **params):
        p = dict(DEFAULT_PARAMS)
        p.update(params)
        s = scene
        self.scene = s
        self._keep = []

        def k(a, f):
            a = f(a)
            self._keep.append(a)
            return a

        g = s["gravity"]
        self.fparams = k([s["dt"], s["dhat"], p.get("kappa", s["kappa"]), g[0], g[1], g[2],
                          p.get("newton_tol", s["newton_tol"]), p["pcg_tol"], p["gap_s"]], _f64)
        nn_guess = len(s["rest_pos"]) + 4 * len(s["body_mass"])
        pcg_max = p["pcg_max"] or 10 * 3 * nn_guess
        self.iparams = k([pcg_max, p["newton_max"], p["ls_max"], p["barrier_form"], p["ccd_max_iter"]], _i32)
        L = lib()
        self.h = L.or_create(
            ctypes.c_int(len(s["rest_pos"])), _dp(k(s["rest_pos"], _f64)), _ip(k(s["vert_body"], _i32)),
            ctypes.c_int(len(s["fixed"])), _ip(k(s["fixed"], _i32)), _dp(k(s["fixed_vel"], _f64)),
            ctypes.c_int(len(s["tets"])), _ip(k(s["tets"], _i32)), _dp(k(s["tet_E"], _f64)), _dp(k(s["tet_nu"], _f64)),
            _dp(k(s["tet_rho"], _f64)),
            ctypes.c_int(len(s["tris"])), _ip(k(s["tris"], _i32)), _dp(k(s["tri_E"], _f64)), _dp(k(s["tri_nu"], _f64)),
            _dp(k(s["tri_thick"], _f64)), _dp(k(s["tri_rho"], _f64)),
            ctypes.c_int(len(s["hinges"])), _ip(k(s["hinges"], _i32)), _dp(k(s["hinge_kb"], _f64)),
            ctypes.c_int(len(s["body_mass"])), _dp(k(s["body_mass"], _f64)), _dp(k(s["body_vol"], _f64)),
            _dp(k(s["body_kappa"], _f64)),
            ctypes.c_int(len(s["surf_tris"])), _ip(k(s["surf_tris"], _i32)),
            ctypes.c_int(len(s["surf_edges"])), _ip(k(s["surf_edges"], _i32)),
            ctypes.c_int(len(s["surf_verts"])), _ip(k(s["surf_verts"], _i32)),
            ctypes.c_int(len(s["planes"])), _dp(k(s["planes"], _f64)),
            _dp(self.fparams), _ip(self.iparams))
        self.h = ctypes.c_void_p(self.h)
        if int(s.get("cloth_model", 0)) == 1:
            L.or_set_cloth_model(self.h, ctypes.c_int(1), _dp(k(s["tri_shear"], _f64)))
        if len(s.get("embed_verts", ())):
            L.or_set_embedding(self.h, ctypes.c_int(len(s["embed_verts"])), _ip(k(s["embed_verts"], _i32)),
                               _ip(k(s["embed_cage"], _i32)), _dp(k(s["embed_w"], _f64)))
        self.nn = L.or_num_nodes(self.h)
        self.nfree = L.or_num_free(self.h)
        self.nv = len(s["rest_pos"])

    def __del__(self):
        try:
            lib().or_destroy(self.h)
        except Exception:
            pass

    def vertex_info(self):
        vnode = np.zeros(self.nv, np.int32)
        vr = np.zeros((self.nv, 3))
        vm = np.zeros(self.nv)
        lib().or_vertex_info(self.h, _ip(vnode), _dp(vr), _dp(vm))
        return vnode, vr, vm

    def initial_state(self):
        x = np.zeros((self.nn, 3))
        v = np.zeros((self.nn, 3))
        lib().or_initial_state(self.h, _dp(_f64(self.scene["vel0"])), _dp(x), _dp(v))
        return x, v

    def positions(self, x):
        P = np.zeros((self.nv, 3))
        lib().or_vertex_positions(self.h, _dp(_f64(x)), _dp(P))
        return P

    def xtilde(self, x, v):
        out = np.zeros((self.nn, 3))
        lib().or_xtilde(self.h, _dp(_f64(x)), _dp(_f64(v)), _dp(out))
        return out

    def set_fixed_positions(self, P):
        lib().or_set_fixed_positions(self.h, _dp(_f64(P)))

    def fixed_positions(self):
        P = np.zeros((self.nv, 3))
        lib().or_get_fixed_positions(self.h, _dp(P))
        return P

    def pairs(self, x, brute=False, cap=1 << 22):
        npt, nee, npg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pt = np.zeros((cap, 3), np.int32)
        ee = np.zeros((cap, 3), np.int32)
        pg = np.zeros((cap, 3), np.int32)
        rc = lib().or_detect_pairs(self.h, _dp(_f64(x)), ctypes.c_int(int(brute)), ctypes.c_int(cap), _ip(pt),
                                   ctypes.byref(npt), _ip(ee), ctypes.byref(nee), _ip(pg), ctypes.byref(npg))
        if rc != 0:
            raise RuntimeError("pair capacity exceeded")
        return pt[:npt.value].copy(), ee[:nee.value].copy(), pg[:npg.value].copy()

    def energy(self, x, xtil, brute=False, terms=False):
        t = np.zeros(6)
        E = lib().or_energy(self.h, _dp(_f64(x)), _dp(_f64(xtil)), ctypes.c_int(int(brute)), _dp(t))
        return (E, t) if terms else E

    def assemble(self, x, xtil, brute=False, project=True):
        lib().or_assemble(self.h, _dp(_f64(x)), _dp(_f64(xtil)), ctypes.c_int(int(brute)), ctypes.c_int(int(project)))
        g = np.zeros((self.nn, 3))
        lib().or_export_grad(self.h, _dp(g))
        return g

    def bsr(self, which):
        """(rowptr, col, vals (nnzb,3,3), diag (nn,3,3)) of the last assembly; which 0 static, 1 dynamic."""
        nnzb = ctypes.c_int()
        lib().or_export_bsr(ctypes.c_int(which), ctypes.byref(nnzb), None, None, None, None)
        rowptr = np.zeros(self.nn + 1, np.int32)
        col = np.zeros(max(nnzb.value, 1), np.int32)
        vals = np.zeros((max(nnzb.value, 1), 9))
        diag = np.zeros((self.nn, 9))
        lib().or_export_bsr(ctypes.c_int(which), ctypes.byref(nnzb), _ip(rowptr), _ip(col), _dp(vals), _dp(diag))
        n = nnzb.value
        return rowptr, col[:n].copy(), vals[:n].reshape(n, 3, 3).copy(), diag.reshape(-1, 3, 3)

    def dense_hessian(self):
        n = self.nn
        H = np.zeros((3 * n, 3 * n))
        for which in (0, 1):
            rowptr, col, vals, diag = self.bsr(which)
            for r in range(n):
                H[3 * r:3 * r + 3, 3 * r:3 * r + 3] += diag[r]
                for q in range(rowptr[r], rowptr[r + 1]):
                    c = col[q]
                    H[3 * r:3 * r + 3, 3 * c:3 * c + 3] += vals[q]
                    H[3 * c:3 * c + 3, 3 * r:3 * r + 3] += vals[q].T
        return H

    def spmv(self, x):
        y = np.zeros((self.nn, 3))
        lib().or_spmv(self.h, _dp(_f64(x)), _dp(y))
        return y

    def set_tet_young(self, E):
        """Per-tet Young's moduli (Poisson ratios kept)."""
        lib().or_set_tet_young(self.h, _dp(_f64(E)))

    def adjoint_step(self, xt, vt, xnext, xbar, vbar, tol=1e-12, maxit=100000):
        """One reverse step of the implicit-function adjoint (form 2).  Returns
        (dL/dx_t, dL/dv_t, dL/dE increment per tet, PCG iterations, status)."""
        xp = np.zeros((self.nn, 3))
        vp = np.zeros((self.nn, 3))
        Eb = np.zeros(len(self.scene["tets"]))
        it = ctypes.c_int()
        rc = lib().or_adjoint_step(self.h, _dp(_f64(xt)), _dp(_f64(vt)), _dp(_f64(xnext)), _dp(_f64(xbar)),
                                   _dp(_f64(vbar)), ctypes.c_double(tol), ctypes.c_int(maxit), _dp(xp), _dp(vp),
                                   _dp(Eb), ctypes.byref(it))
        return xp, vp, Eb, it.value, rc

    def rollout(self, x0, v0, n_steps, brute=False):
        """Forward rollout; returns the list of (x_t, v_t) for t = 0..n_steps and the statuses."""
        x, v = _f64(x0).copy(), _f64(v0).copy()
        states = [(x.copy(), v.copy())]
        rcs = []
        for _ in range(n_steps):
            x, v, rc, _st = self.step(x, v, brute=brute)
            states.append((x.copy(), v.copy()))
            rcs.append(rc)
        return states, rcs

    def rollout_adjoint(self, states, xbar_T, vbar_T, tol=1e-12):
        """Reverse pass over a rollout: dL/dx_0, dL/dv_0, dL/dE per tet."""
        xbar, vbar = _f64(xbar_T).copy(), _f64(vbar_T).copy()
        Ebar = np.zeros(len(self.scene["tets"]))
        for t in range(len(states) - 2, -1, -1):
            xt, vt = states[t]
            xbar, vbar, Eb, _it, rc = self.adjoint_step(xt, vt, states[t + 1][0], xbar, vbar, tol=tol)
            if rc != 0:
                raise RuntimeError(f"adjoint PCG did not converge at step {t}")
            Ebar += Eb
        return xbar, vbar, Ebar

    def pcg(self, rhs, tol=1e-4, maxit=100000):
        x = np.zeros((self.nn, 3))
        it = ctypes.c_int()
        rc = lib().or_pcg(self.h, _dp(_f64(rhs)), _dp(x), ctypes.c_double(tol), ctypes.c_int(maxit), ctypes.byref(it))
        return x, it.value, rc

    def set_kappa_adaptive(self, on=True, kappa_min=None, kappa_max=None, dmin=None):
        """Adaptive barrier stiffness (reading c5): chosen at each step's start,
        frozen for the step.  The first step that starts with contact pairs
        balances the barrier gradient against the rest, clamped to
        [kappa_min, kappa_max]; later steps double kappa (up to kappa_max) when
        the smallest pair distance is below ``dmin`` (default dhat / 10) and
        smaller than at the previous step's start.  kappa_min None: the
        stiffness at which the barrier holds an average vertex's weight at
        dhat / 2; kappa_max None: 1e4 kappa_min."""
        d = self.scene["dhat"] / 10.0 if dmin is None else dmin
        lib().or_set_kappa_adaptive(self.h, ctypes.c_int(int(on)), ctypes.c_double(kappa_min or 0.0),
                                    ctypes.c_double(kappa_max or 0.0), ctypes.c_double(d))

    def kappa_bounds(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        lib().or_get_kappa_bounds(self.h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    @property
    def kappa(self):
        return lib().or_get_kappa(self.h)

    def ccd_bound(self, x, direction, brute=False):
        return lib().or_ccd_bound(self.h, _dp(_f64(x)), _dp(_f64(direction)), ctypes.c_int(int(brute)))

    def step(self, x, v, brute=False):
        """One implicit time step in place on copies; returns (x, v, rc, stats dict)."""
        x = _f64(x).copy()
        v = _f64(v).copy()
        st = np.zeros(9)
        rc = lib().or_step(self.h, _dp(x), _dp(v), ctypes.c_int(int(brute)), _dp(st))
        keys = ["newton_iters", "pcg_iters", "alpha", "p_inf", "n_pt", "n_ee", "n_pg", "ls_fail", "kappa"]
        return x, v, rc, dict(zip(keys, st.tolist()))


def num_threads():
    return lib().or_num_threads()
