"""Seeded synthetic scene generators for the IPC Newton hot path.

This module produces *inputs only*: rest positions, connectivity, material
parameters, fixed vertices, affine-body membership, collision surfaces and
planes.  It holds none of the method's arithmetic (no deformation gradients,
no rest-shape inverses, no masses, no energies); both the CUDA library and the
CPU oracle derive those themselves from what is returned here.

A scene is a plain ``dict`` of numpy arrays (float64 / int32) plus scalar
parameters.  Index arrays are 0-based.  Keys:

  rest_pos  (nv,3)   undeformed, world-placed vertex positions (initial state)
  vel0      (nv,3)   initial vertex velocities
  vert_body (nv,)    -1 for a free / fixed vertex, else affine body id
  fixed     (nf,)    ids of vertices with prescribed (Dirichlet) positions
  fixed_vel (nf,3)   prescribed velocity of those vertices
  tets      (nt,4)   tet2v, positively oriented;  tet_E, tet_nu, tet_rho (nt,)
  tris      (nc,3)   cloth (membrane) triangles;  tri_E, tri_nu, tri_thick, tri_rho
  hinges    (nh,4)   (e0, e1, a, b): shared edge (e0,e1), opposite vertices a, b;
                     hinge_kb (nh,)
  body_mass, body_vol, body_kappa (nb,)   affine-body mass, volume, orthogonality
                     stiffness
  surf_tris (ns,3), surf_edges (ne,2), surf_verts (nsv,)   collision surface
  planes    (np,4)   (nx, ny, nz, c): half-space n.x >= c is free
  dt, dhat, kappa, gravity (3,), n_steps, newton_tol   run parameters
  name      str

The geometric recipes follow the five synthetic workloads that stand in for the
paper's bunny scenes: stacked cubes, sphere + cloth + affine boxes, a pile of 64
tori, a clamped beam, and batches of soft grippers.
"""
import numpy as np

__all__ = [
    "hex_grid", "kuhn_tets", "voxel_tets", "boundary_faces", "unique_edges",
    "cloth_grid", "cloth_hinges", "box_surface", "random_rotations",
    "cubes_scene", "tori_scene", "mixed_scene", "beam_scene", "gripper_batch",
    "merge_meshes", "finalize_scene", "scene_by_name",
]


# --------------------------------------------------------------------------
# mesh primitives
# --------------------------------------------------------------------------
def hex_grid(nx, ny, nz, h, origin=(0.0, 0.0, 0.0)):
    """Vertices of an (nx+1)x(ny+1)x(nz+1) lattice with spacing h (x fastest)."""
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # order: x fastest, then y, then z  -> index = i + (nx+1)*(j + (ny+1)*k)
    ii = ii.transpose(2, 1, 0).ravel()
    jj = jj.transpose(2, 1, 0).ravel()
    kk = kk.transpose(2, 1, 0).ravel()
    v = np.stack([ii, jj, kk], axis=1).astype(np.float64) * h + np.asarray(origin, np.float64)
    return v


# The six Kuhn (Freudenthal) tets of a unit cube: every path from corner 000 to
# corner 111 that steps along the three axes in some order.  The split is
# conforming across neighbouring cubes of a lattice.
_KUHN_PATHS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def kuhn_tets(nx, ny, nz, keep=None):
    """Tet connectivity of the Kuhn split of an nx*ny*nz hex lattice.

    keep: optional boolean array (nx,ny,nz) selecting which hexes to split.
    Returns (nt,4) int array, vertex ids in hex_grid numbering, positively
    oriented (the orientation fix uses only the sign of the permutation).
    """
    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    out = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if keep is not None and not keep[i, j, k]:
                    continue
                for perm in _KUHN_PATHS:
                    c = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in perm:
                        c[ax] += 1
                        path.append(vid(i + c[0], j + c[1], k + c[2]))
                    out.append(path)
    t = np.asarray(out, dtype=np.int64).reshape(-1, 4)
    # path (0,1,2) = 000,100,110,111 has det([e1, e1+e2, e1+e2+e3]) = +1; an odd
    # permutation of the axes flips the sign.  Swap the last two ids for those.
    parity = np.array([0, 1, 1, 0, 0, 1], dtype=bool)  # odd permutations of (0,1,2)
    n_per = 6
    if len(t):
        reps = np.tile(parity, len(t) // n_per)
        t[reps, 2], t[reps, 3] = t[reps, 3].copy(), t[reps, 2].copy()
    return t


def _compact(verts, tets):
    used = np.unique(tets)
    remap = -np.ones(len(verts), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return verts[used], remap[tets]


def voxel_tets(inside, lo, hi, h):
    """Voxelise an implicit shape: keep lattice hexes whose centre is inside.

    inside: callable (m,3) -> bool (m,).  lo, hi: bounding box corners.
    Returns (verts (nv,3), tets (nt,4)) with unused lattice vertices removed.
    """
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    n = np.maximum(np.ceil((hi - lo) / h).astype(int), 1)
    # centre the lattice on the box
    origin = (lo + hi) / 2 - n * h / 2
    ci = (np.arange(n[0]) + 0.5) * h + origin[0]
    cj = (np.arange(n[1]) + 0.5) * h + origin[1]
    ck = (np.arange(n[2]) + 0.5) * h + origin[2]
    C = np.stack(np.meshgrid(ci, cj, ck, indexing="ij"), axis=-1)
    keep = inside(C.reshape(-1, 3)).reshape(n[0], n[1], n[2])
    v = hex_grid(n[0], n[1], n[2], h, origin)
    t = kuhn_tets(n[0], n[1], n[2], keep)
    return _compact(v, t)


# outward faces of a positively oriented tet (v0,v1,v2,v3)
_TET_FACES = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])


def boundary_faces(tets):
    """Faces used by exactly one tet, oriented outward."""
    f = tets[:, _TET_FACES].reshape(-1, 3)
    key = np.sort(f, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    return f[cnt[inv] == 1]


def unique_edges(tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def cloth_grid(n, size, origin=(0.0, 0.0, 0.0)):
    """n x n vertex grid in the x-z plane (y = origin[1]), 2(n-1)^2 triangles."""
    s = np.linspace(0.0, size, n)
    X, Z = np.meshgrid(s, s, indexing="xy")   # row-major: z rows, x columns
    v = np.stack([X.ravel(), np.zeros(n * n), Z.ravel()], axis=1) + np.asarray(origin, np.float64)
    tris = []
    for r in range(n - 1):
        for c in range(n - 1):
            a = r * n + c
            b = a + 1
            d = a + n
            e = d + 1
            # alternate the diagonal for a less anisotropic mesh
            if (r + c) % 2 == 0:
                tris.append([a, d, b]); tris.append([b, d, e])
            else:
                tris.append([a, d, e]); tris.append([a, e, b])
    return v, np.asarray(tris, dtype=np.int64)


def cloth_hinges(tris):
    """Interior edges with their two opposite vertices: (e0, e1, a, b)."""
    edges = {}
    for t in tris:
        for k in range(3):
            i, j, o = t[k], t[(k + 1) % 3], t[(k + 2) % 3]
            key = (min(i, j), max(i, j))
            edges.setdefault(key, []).append((i, j, o))
    out = []
    for key, lst in edges.items():
        if len(lst) == 2:
            (i, j, a), (_, _, b) = lst
            out.append([i, j, a, b])
    out.sort()
    return np.asarray(out, dtype=np.int64).reshape(-1, 4)


def box_surface(size, center):
    """Closed box: 8 corners, 12 outward triangles."""
    c = np.asarray(center, np.float64)
    hs = size / 2
    v = np.array([[x, y, z] for z in (-hs, hs) for y in (-hs, hs) for x in (-hs, hs)], np.float64) + c
    # corner index = x + 2y + 4z
    f = np.array([
        [0, 2, 1], [1, 2, 3],      # z-
        [4, 5, 6], [5, 7, 6],      # z+
        [0, 1, 4], [1, 5, 4],      # y-
        [2, 6, 3], [3, 6, 7],      # y+
        [0, 4, 2], [2, 4, 6],      # x-
        [1, 3, 5], [3, 7, 5],      # x+
    ], dtype=np.int64)
    return v, f


def random_rotations(rng, n):
    """Uniformly distributed rotations from uniform unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    q = np.stack([
        np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
        np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
        np.sqrt(u1) * np.sin(2 * np.pi * u3),
        np.sqrt(u1) * np.cos(2 * np.pi * u3)], axis=1)  # (x, y, z, w)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


# --------------------------------------------------------------------------
# scene assembly
# --------------------------------------------------------------------------
def _empty_parts():
    return dict(verts=[], vel=[], body=[], tets=[], tet_E=[], tet_nu=[], tet_rho=[],
                tris=[], tri_E=[], tri_nu=[], tri_thick=[], tri_rho=[], tri_shear=[], hinges=[], hinge_kb=[],
                surf_tris=[], fixed=[], fixed_vel=[], body_mass=[], body_vol=[], body_kappa=[], nv=0, nb=0)


def _add_soft(parts, verts, tets, E, nu, rho, vel=None, surface=True):
    off = parts["nv"]
    nv = len(verts)
    parts["verts"].append(verts)
    parts["vel"].append(np.zeros((nv, 3)) if vel is None else vel)
    parts["body"].append(-np.ones(nv, dtype=np.int64))
    parts["tets"].append(tets + off)
    nt = len(tets)
    parts["tet_E"].append(np.broadcast_to(np.asarray(E, np.float64), (nt,)).copy())
    parts["tet_nu"].append(np.full(nt, nu, np.float64))
    parts["tet_rho"].append(np.full(nt, rho, np.float64))
    if surface:
        parts["surf_tris"].append(boundary_faces(tets) + off)
    parts["nv"] += nv
    return off


def _add_embedded_surface(parts, verts, faces, cage_off, cage_origin, cage_h, cage_dims):
    """A surface mesh embedded in a hex cage (the cage parameterisation): every
    vertex is tied to the 8 corners of the cage cell that encloses it by
    trilinear weights; vert_body -2, no mass and no element of its own."""
    nx, ny, nz = cage_dims
    off = parts["nv"]
    nv = len(verts)
    parts["verts"].append(verts)
    parts["vel"].append(np.zeros((nv, 3)))
    parts["body"].append(np.full(nv, -2, dtype=np.int64))
    parts["surf_tris"].append(faces + off)
    u = (verts - np.asarray(cage_origin)) / cage_h
    cell = np.clip(np.floor(u).astype(np.int64), 0, np.array([nx - 1, ny - 1, nz - 1]))
    f = u - cell
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
    cage = np.zeros((nv, 8), np.int64)
    w = np.zeros((nv, 8))
    q = 0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                cage[:, q] = cage_off + vid(cell[:, 0] + di, cell[:, 1] + dj, cell[:, 2] + dk)
                w[:, q] = ((f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) *
                           (f[:, 2] if dk else 1 - f[:, 2]))
                q += 1
    parts.setdefault("embed_verts", []).append(np.arange(off, off + nv))
    parts.setdefault("embed_cage", []).append(cage)
    parts.setdefault("embed_w", []).append(w)
    parts["nv"] += nv
    return off


def _add_cloth(parts, verts, tris, E, nu, thick, rho, kb, shear=0.0):
    off = parts["nv"]
    nv = len(verts)
    parts["verts"].append(verts)
    parts["vel"].append(np.zeros((nv, 3)))
    parts["body"].append(-np.ones(nv, dtype=np.int64))
    parts["tris"].append(tris + off)
    nc = len(tris)
    parts["tri_E"].append(np.full(nc, E)); parts["tri_nu"].append(np.full(nc, nu))
    parts["tri_thick"].append(np.full(nc, thick)); parts["tri_rho"].append(np.full(nc, rho))
    parts["tri_shear"].append(np.full(nc, shear))
    h = cloth_hinges(tris)
    parts["hinges"].append(h + off)
    parts["hinge_kb"].append(np.full(len(h), kb))
    parts["surf_tris"].append(tris + off)
    parts["nv"] += nv
    return off


def _add_body(parts, verts, faces, mass, vol, kappa):
    off = parts["nv"]
    nv = len(verts)
    b = parts["nb"]
    parts["verts"].append(verts)
    parts["vel"].append(np.zeros((nv, 3)))
    parts["body"].append(np.full(nv, b, dtype=np.int64))
    parts["surf_tris"].append(faces + off)
    parts["body_mass"].append(mass); parts["body_vol"].append(vol); parts["body_kappa"].append(kappa)
    parts["nv"] += nv
    parts["nb"] += 1
    return off


def _cat(lst, shape_tail, dtype):
    if not lst:
        return np.zeros((0,) + shape_tail, dtype=dtype)
    return np.ascontiguousarray(np.concatenate(lst, axis=0).astype(dtype))


def finalize_scene(parts, name, dt, dhat, kappa, n_steps, planes, gravity=(0.0, -9.81, 0.0), newton_tol_rel=1e-5):
    s = {}
    s["name"] = name
    s["rest_pos"] = _cat(parts["verts"], (3,), np.float64)
    s["vel0"] = _cat(parts["vel"], (3,), np.float64)
    s["vert_body"] = _cat(parts["body"], (), np.int32)
    s["fixed"] = _cat([np.asarray(f, np.int64) for f in parts["fixed"]], (), np.int32)
    s["fixed_vel"] = _cat([np.asarray(f, np.float64).reshape(-1, 3) for f in parts["fixed_vel"]], (3,), np.float64)
    s["tets"] = _cat(parts["tets"], (4,), np.int32)
    for k in ("tet_E", "tet_nu", "tet_rho", "tri_E", "tri_nu", "tri_thick", "tri_rho", "tri_shear", "hinge_kb"):
        s[k] = _cat(parts[k], (), np.float64)
    s["tris"] = _cat(parts["tris"], (3,), np.int32)
    s["hinges"] = _cat(parts["hinges"], (4,), np.int32)
    s["body_mass"] = np.asarray(parts["body_mass"], np.float64)
    s["body_vol"] = np.asarray(parts["body_vol"], np.float64)
    s["body_kappa"] = np.asarray(parts["body_kappa"], np.float64)
    st = _cat(parts["surf_tris"], (3,), np.int32)
    s["surf_tris"] = st
    s["surf_edges"] = unique_edges(st).astype(np.int32) if len(st) else np.zeros((0, 2), np.int32)
    s["surf_verts"] = np.unique(st).astype(np.int32) if len(st) else np.zeros((0,), np.int32)
    s["planes"] = np.asarray(planes, np.float64).reshape(-1, 4)
    s["cloth_model"] = int(parts.get("cloth_model", 0))
    s["embed_verts"] = _cat(parts.get("embed_verts", []), (), np.int32)
    s["embed_cage"] = _cat(parts.get("embed_cage", []), (8,), np.int32)
    s["embed_w"] = _cat(parts.get("embed_w", []), (8,), np.float64)
    s["dt"] = float(dt)
    s["dhat"] = float(dhat)
    s["kappa"] = float(kappa)
    s["gravity"] = np.asarray(gravity, np.float64)
    s["n_steps"] = int(n_steps)
    lo, hi = s["rest_pos"].min(0), s["rest_pos"].max(0)
    s["bbox_diag"] = float(np.linalg.norm(hi - lo))
    s["newton_tol"] = float(newton_tol_rel * dt * s["bbox_diag"])
    return s


def merge_meshes(*a, **k):  # kept for API symmetry; scenes are merged via the parts helpers
    raise NotImplementedError


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def cubes_scene(n=4, side=0.1, gap=0.002, shift=0.01, E=1e5, nu=0.4, rho=1000.0,
                dt=0.01, dhat=1e-3, kappa=1e4, n_steps=50):
    """Two stacked soft cubes (n^3 hexes, 6 tets each) above a ground plane y=0."""
    parts = _empty_parts()
    h = side / n
    t = kuhn_tets(n, n, n)
    v_bot = hex_grid(n, n, n, h, (0.0, gap, 0.0))
    v_top = hex_grid(n, n, n, h, (shift, gap + side + gap, 0.0))
    _add_soft(parts, v_bot, t, E, nu, rho)
    _add_soft(parts, v_top, t, E, nu, rho)
    return finalize_scene(parts, "cubes", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def _torus_inside(R, r):
    def f(p):
        q = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2) - R
        return q * q + p[:, 2] ** 2 <= r * r
    return f


def torus_mesh(R=0.08, r=0.03, h=0.008):
    return voxel_tets(_torus_inside(R, r), (-(R + r), -(R + r), -r), (R + r, R + r, r), h)


def sphere_mesh(radius, h):
    return voxel_tets(lambda p: (p * p).sum(1) <= radius * radius, (-radius,) * 3, (radius,) * 3, h)


def cube_mesh(side, h):
    n = max(1, int(round(side / h)))
    return hex_grid(n, n, n, side / n, (-side / 2,) * 3), kuhn_tets(n, n, n)


def tori_scene(nx=4, ny=4, nz=4, spacing=0.24, R=0.08, r=0.03, h=0.008, seed=0, box=1.0,
               nu=0.4, rho=1000.0, dt=0.01, dhat=1e-3, kappa=1e4, n_steps=100):
    """64 randomly oriented Neo-Hookean tori on a lattice inside a 1 m box."""
    rng = np.random.default_rng(seed)
    tv, tt = torus_mesh(R, r, h)
    n = nx * ny * nz
    Rs = random_rotations(rng, n)
    Es = np.exp(rng.uniform(np.log(1e4), np.log(1e6), n))
    parts = _empty_parts()
    margin = [(box - spacing * (n_ - 1)) / 2 for n_ in (nx, ny, nz)]
    idx = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = np.array([margin[0] + i * spacing, margin[1] + j * spacing, margin[2] + k * spacing])
                v = tv @ Rs[idx].T + c
                _add_soft(parts, v, tt, Es[idx], nu, rho)
                idx += 1
    planes = [[0, 1, 0, 0], [1, 0, 0, 0], [-1, 0, 0, -box], [0, 0, 1, 0], [0, 0, -1, -box]]
    return finalize_scene(parts, "tori", dt, dhat, kappa, n_steps, planes=planes)


def mixed_scene(sphere_r=0.1, sphere_h=0.0108, cloth_n=101, cloth_size=1.0, n_boxes=16, box_size=0.04,
                seed=0, dt=0.005, dhat=5e-4, kappa=1e4, n_steps=200):
    """Soft sphere + StVK cloth + 16 affine boxes (every cross-parameterisation pair)."""
    parts = _empty_parts()
    sv, st = sphere_mesh(sphere_r, sphere_h)
    sv = sv + np.array([0.0, 1e-3 - sv[:, 1].min(), 0.0])  # resting 1 mm above the ground
    _add_soft(parts, sv, st, 5e4, 0.4, 1000.0)
    top = sv[:, 1].max()
    thick = 1e-3
    E_c, nu_c = 1e6, 0.3
    kb = E_c * thick ** 3 / (24 * (1 - nu_c ** 2))
    cv, ct = cloth_grid(cloth_n, cloth_size, (-cloth_size / 2, top + 0.01, -cloth_size / 2))
    _add_cloth(parts, cv, ct, E_c, nu_c, thick, 1000.0, kb)
    side = int(round(np.sqrt(n_boxes)))
    for b in range(n_boxes):
        i, k = b % side, b // side
        c = np.array([(i - (side - 1) / 2) * 0.1, top + 0.01 + 0.05 + box_size / 2, (k - (side - 1) / 2) * 0.1])
        bv, bf = box_surface(box_size, c)
        _add_body(parts, bv, bf, mass=1000.0 * box_size ** 3, vol=box_size ** 3, kappa=1e8)
    return finalize_scene(parts, "mixed", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def union_contact_scene(gap=3e-4, dhat=1e-3, kappa=1e4, dt=0.01, seed=0):
    """A small scene where every UNION combination is in contact at rest.

    Box A (affine) rests ``gap`` above the ground; box B (affine, turned 20
    degrees about y) sits ``gap`` above A, so their faces and crossing edges
    form body-body point-triangle and edge-edge pairs; a 3x3 cloth lies
    ``gap`` above B (free vertex on body triangle) and box C (affine) lies
    ``gap`` above the cloth (body vertex on free triangle); a one-hex soft
    block (6 tets) stands ``gap`` from A's +x face and ``gap`` above the ground
    (free vertex on body triangle, free point-ground).
    """
    parts = _empty_parts()
    sa, sb, sc = 0.04, 0.03, 0.008
    av, af = box_surface(sa, (0.0, gap + sa / 2, 0.0))
    _add_body(parts, av, af, mass=1000.0 * sa ** 3, vol=sa ** 3, kappa=1e8)
    c = np.cos(np.radians(20.0)); sn = np.sin(np.radians(20.0))
    Ry = np.array([[c, 0.0, sn], [0.0, 1.0, 0.0], [-sn, 0.0, c]])
    b_c = np.array([0.002, gap + sa + gap + sb / 2, 0.001])
    bv, bf = box_surface(sb, (0.0, 0.0, 0.0))
    _add_body(parts, bv @ Ry.T + b_c, bf, mass=1000.0 * sb ** 3, vol=sb ** 3, kappa=1e8)
    top_b = b_c[1] + sb / 2
    thick, E_c, nu_c = 1e-3, 1e6, 0.3
    kb = E_c * thick ** 3 / (24 * (1 - nu_c ** 2))
    cs = 0.016
    cv, ct = cloth_grid(3, cs, (b_c[0] - cs / 2, top_b + gap, b_c[2] - cs / 2))
    _add_cloth(parts, cv, ct, E_c, nu_c, thick, 1000.0, kb)
    cvv, cf = box_surface(sc, (b_c[0] + 0.001, top_b + 2 * gap + sc / 2, b_c[2] - 0.001))
    _add_body(parts, cvv, cf, mass=1000.0 * sc ** 3, vol=sc ** 3, kappa=1e8)
    hs = 0.015
    hv = hex_grid(1, 1, 1, hs, (sa / 2 + gap, gap, -hs / 2))
    _add_soft(parts, hv, kuhn_tets(1, 1, 1), 1e5, 0.4, 1000.0)
    return finalize_scene(parts, "union_contact", dt, dhat, kappa, 1, planes=[[0, 1, 0, 0]])


def blob_mesh(h, radius=0.05, seed=0):
    """A voxelised lumpy blob (the stand-in for the bunny of the paper's cloth
    scenes): a sphere of the given radius with two smaller spheres attached."""
    rng = np.random.default_rng(seed)
    centres = [(0.0, 0.0, 0.0), (0.6 * radius, 0.55 * radius, 0.0), (-0.5 * radius, 0.3 * radius, 0.45 * radius)]
    radii = [radius, 0.55 * radius, 0.45 * radius * (1.0 + 0.1 * rng.random())]

    def inside(p):
        ok = np.zeros(len(p), bool)
        for c, r in zip(centres, radii):
            ok |= np.linalg.norm(p - np.asarray(c), axis=1) <= r
        return ok

    lo = np.full(3, -1.2 * radius)
    hi = np.full(3, 1.2 * radius)
    return voxel_tets(inside, lo, hi, h)


def bw_cloth_scene(cloth_n=101, cloth_size=1.0, layers=1, blob_h=0.01, blob_radius=0.12, seed=0, dt=0.01,
                   dhat=1e-3, kappa=1e4, n_steps=200):
    """The shape of the paper's first cloth benchmark (Sec. "Cloths on Bunny on
    Cloth", Table 1) with synthetic inputs: a voxelised soft blob (stable
    Neo-Hookean, E 10259 Pa, nu 0.205) held 2 cm above a Baraff-Witkin cloth
    sheet pinned at its four corners (stretch 33570 Pa, shear 100607 Pa,
    bending 0.055, 1 mm thick), and `layers` - 1 more sheets 3 cm apart above
    the blob, free to fall onto it."""
    parts = _empty_parts()
    parts["cloth_model"] = 1
    bv, bt = blob_mesh(blob_h, blob_radius, seed)
    sheet_y = 0.3
    bv = bv + np.array([0.0, sheet_y + 0.02 - bv[:, 1].min(), 0.0])
    _add_soft(parts, bv, bt, 10259.0, 0.205, 1000.0)
    top = bv[:, 1].max()
    for k in range(layers):
        y = sheet_y if k == 0 else top + 0.03 * k
        cv, ct = cloth_grid(cloth_n, cloth_size, (-cloth_size / 2, y, -cloth_size / 2))
        off = _add_cloth(parts, cv, ct, 33570.0, 0.0, 1e-3, 1000.0, 0.055, shear=100607.0)
        if k == 0:
            corners = [0, cloth_n - 1, cloth_n * (cloth_n - 1), cloth_n * cloth_n - 1]
            parts["fixed"].append([off + c for c in corners])
            parts["fixed_vel"].append(np.zeros((4, 3)))
    return finalize_scene(parts, "bw_cloth", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def near_pairs_scene(n_pairs=2000, extent=1.0, size=0.005, dhat=1e-3, speed=0.05, seed=0, dt=0.01, kappa=1e4):
    """Pairs of small free cloth triangles (edges of about `size`) at random
    places up to `extent` from the origin, the second of each pair a slightly
    rotated copy of the first moved by 0.5 to 2.5 dhat in a random direction,
    with random velocities of about `speed`: point-triangle and edge-edge
    distances spread on both sides of dhat at coordinates where single
    precision rounds the most.  A stress input for the contact filters."""
    rng = np.random.default_rng(seed)
    parts = _empty_parts()
    verts, tris, vel = [], [], []
    R = random_rotations(rng, n_pairs)
    for k in range(n_pairs):
        c = rng.uniform(-extent, extent, 3)
        base = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.9, 0.0]]) * size * rng.uniform(0.5, 1.5)
        A = base @ R[k].T + c
        ang = rng.uniform(0.0, 0.3)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        Q = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        o = rng.normal(size=3)
        o *= dhat * rng.uniform(0.5, 2.5) / np.linalg.norm(o)
        ctr = A.mean(0)
        B = (A - ctr) @ Q.T + ctr + o
        for T_ in (A, B):
            tris.append(np.arange(3) + 3 * len(tris))
            verts.append(T_)
            vel.append(np.repeat(rng.normal(size=(1, 3)) * speed, 3, axis=0))
    V = np.concatenate(verts)
    off = _add_cloth(parts, V, np.array(tris), 1e5, 0.3, 1e-3, 1000.0, 0.0)
    parts["vel"][-1] = np.concatenate(vel)
    return finalize_scene(parts, "near_pairs", dt, dhat, kappa, 1, planes=np.zeros((0, 4)))


def caged_blob_scene(blob_h=0.01, blob_radius=0.05, cage_h=0.025, E=3.17e4, nu=0.226, rho=1000.0, lift=3e-4,
                     with_box=True, seed=0, dt=0.01, dhat=1e-3, kappa=1e4, n_steps=150):
    """The cage example's shape (Sec. "Caged Bunny", Table "Caged Bunny"; the
    bunny replaced by a voxelised blob): the blob's boundary surface, embedded
    by trilinear weights in a uniform hex cage of spacing cage_h whose cells
    are split into 6 stable Neo-Hookean tets each (E 31.7 kPa, nu 0.226); the
    cage vertices are free and do not collide, the embedded surface does.  The
    surface's lowest point starts `lift` above the ground; with_box adds an
    affine box resting `lift` above the surface's highest point."""
    parts = _empty_parts()
    bv, bt = blob_mesh(blob_h, blob_radius, seed)
    faces = boundary_faces(bt)
    used = np.unique(faces)
    remap = -np.ones(len(bv), np.int64)
    remap[used] = np.arange(len(used))
    sv, sf = bv[used], remap[faces]
    sv = sv + np.array([0.0, lift - sv[:, 1].min(), 0.0])
    lo, hi = sv.min(0) - 1e-3, sv.max(0) + 1e-3
    dims = np.maximum(np.ceil((hi - lo) / cage_h).astype(int), 1)
    cv = hex_grid(dims[0], dims[1], dims[2], cage_h, lo)
    ct = kuhn_tets(dims[0], dims[1], dims[2])
    coff = _add_soft(parts, cv, ct, E, nu, rho, surface=False)
    _add_embedded_surface(parts, sv, sf, coff, lo, cage_h, tuple(dims))
    if with_box:  # an affine box resting on the surface's highest point
        size = 0.03
        top = sv[np.argmax(sv[:, 1])]
        bx, bf = box_surface(size, (top[0] + 0.004, top[1] + lift + size / 2, top[2] - 0.003))
        _add_body(parts, bx, bf, mass=1000.0 * size ** 3, vol=size ** 3, kappa=1e8)
    return finalize_scene(parts, "caged_blob", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def beam_scene(nx=52, ny=8, nz=8, length=1.0, width=0.1, lift=0.02, seed=0, dt=0.01, dhat=1e-3,
               kappa=1e4, n_steps=20, rho=1000.0, nu=0.4):
    """Clamped beam (x=0 face fixed) with log-uniform per-tet E and N(0,0.1) velocities."""
    rng = np.random.default_rng(seed)
    v = hex_grid(nx, ny, nz, 1.0, (0.0, 0.0, 0.0)) * np.array([length / nx, width / ny, width / nz])
    v[:, 1] += lift
    t = kuhn_tets(nx, ny, nz)
    E = np.exp(rng.uniform(np.log(1e4), np.log(1e5), len(t)))
    vel = rng.normal(0.0, 0.1, size=(len(v), 3))
    parts = _empty_parts()
    _add_soft(parts, v, t, E, nu, rho, vel=vel)
    fixed = np.nonzero(v[:, 0] <= 1e-12)[0]
    parts["fixed"].append(fixed)
    parts["fixed_vel"].append(np.zeros((len(fixed), 3)))
    parts["vel"][0][fixed] = 0.0
    return finalize_scene(parts, "beam", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def gripper_scene(n_tets_target, rng, dt=0.01, dhat=1e-3, kappa=1e4, n_steps=100):
    """One soft two-finger gripper closing on a random deformable object."""
    kind = rng.integers(0, 3)
    E_obj = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
    obj_tets = n_tets_target // 2
    parts = _empty_parts()
    size = 0.05
    if kind == 0:
        vol = 4 / 3 * np.pi * (size / 2) ** 3
        h = (vol / (obj_tets / 6)) ** (1 / 3)
        ov, ot = sphere_mesh(size / 2, h)
    elif kind == 1:
        h = (size ** 3 / (obj_tets / 6)) ** (1 / 3)
        ov, ot = cube_mesh(size, h)
    else:
        R, r = size * 0.35, size * 0.15
        vol = 2 * np.pi ** 2 * R * r * r
        h = (vol / (obj_tets / 6)) ** (1 / 3)
        ov, ot = torus_mesh(R, r, h)
    ov = ov - np.array([0.0, ov[:, 1].min() - 1e-3 - 0.0, 0.0]) * np.array([0, 1, 0])
    ov[:, 1] += 0.0
    _add_soft(parts, ov, ot, E_obj, 0.4, 1000.0)
    # two fingers: box beams on either side in x, gap 5 mm from the object's extent
    fin_tets = n_tets_target // 4
    fl, fw = 0.08, 0.02
    nh = max(1, fin_tets // 6)
    nxf = max(2, int(round((nh * fl * fl / (fw * fw)) ** (1 / 3))))
    nyf = max(1, int(round(nxf * fw / fl)))
    xmin, xmax = ov[:, 0].min(), ov[:, 0].max()
    for side in (-1, 1):
        fv = hex_grid(nyf, nxf, nyf, 1.0) * np.array([fw / nyf, fl / nxf, fw / nyf])
        # fingers stand 2 mm above the ground and reach above the object
        fv = fv + np.array([0.0, 2e-3, -fw / 2])
        if side < 0:
            fv[:, 0] += xmin - 5e-3 - fw
        else:
            fv[:, 0] += xmax + 5e-3
        ft = kuhn_tets(nyf, nxf, nyf)
        off = _add_soft(parts, fv, ft, 2e5, 0.4, 1000.0)
        # root layer (outermost x face) driven inward at 0.02 m/s
        outer = fv[:, 0].min() if side < 0 else fv[:, 0].max()
        root = np.nonzero(np.abs(fv[:, 0] - outer) <= 1e-12)[0] + off
        parts["fixed"].append(root)
        parts["fixed_vel"].append(np.tile([0.02 * -side, 0.0, 0.0], (len(root), 1)))
    return finalize_scene(parts, "gripper", dt, dhat, kappa, n_steps, planes=[[0, 1, 0, 0]])


def gripper_batch(n_scenes=256, lo=1000, hi=20000, seed=0):
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_scenes)).astype(int)
    return [gripper_scene(int(s), rng) for s in sizes]


def concat_scenes(scenes, newton_tol=None):
    """One batch of independent scenes: arrays concatenated with vertex and body
    offsets, ``vert_scene`` the scene of every vertex.  The scenes must share
    dt, dhat, kappa, gravity and planes; the batch's Newton tolerance is the
    smallest of theirs unless given."""
    first = scenes[0]
    for sc in scenes[1:]:
        for k in ("dt", "dhat", "kappa"):
            if sc[k] != first[k]:
                raise ValueError(f"scenes of a batch must share {k}")
        if not (np.array_equal(sc["gravity"], first["gravity"]) and np.array_equal(sc["planes"], first["planes"])):
            raise ValueError("scenes of a batch must share gravity and planes")
    out = {"name": "batch", "planes": first["planes"].copy(), "dt": first["dt"], "dhat": first["dhat"],
           "kappa": first["kappa"], "gravity": first["gravity"].copy(), "n_steps": first["n_steps"]}
    voff, boff = 0, 0
    acc = {k: [] for k in ("rest_pos", "vel0", "vert_body", "fixed", "fixed_vel", "tets", "tet_E", "tet_nu", "tet_rho",
                           "tris", "tri_E", "tri_nu", "tri_thick", "tri_rho", "tri_shear", "hinges", "hinge_kb", "body_mass",
                           "body_vol", "body_kappa", "surf_tris", "surf_edges", "surf_verts", "vert_scene")}
    for k, sc in enumerate(scenes):
        nv = len(sc["rest_pos"])
        for key in ("rest_pos", "vel0", "fixed_vel", "tet_E", "tet_nu", "tet_rho", "tri_E", "tri_nu", "tri_thick",
                    "tri_rho", "tri_shear", "hinge_kb", "body_mass", "body_vol", "body_kappa"):
            acc[key].append(np.asarray(sc.get(key, np.zeros(len(sc["tris"])) if key == "tri_shear" else None)))
        vb = np.asarray(sc["vert_body"]).copy()
        vb[vb >= 0] += boff
        acc["vert_body"].append(vb)
        for key in ("fixed", "tets", "tris", "hinges", "surf_tris", "surf_edges", "surf_verts"):
            acc[key].append(np.asarray(sc[key]) + voff)
        acc["vert_scene"].append(np.full(nv, k, np.int32))
        voff += nv
        boff += len(sc["body_mass"])
    ints = ("vert_body", "fixed", "tets", "tris", "hinges", "surf_tris", "surf_edges", "surf_verts", "vert_scene")
    for key, lst in acc.items():
        out[key] = np.ascontiguousarray(np.concatenate(lst, axis=0).astype(np.int32 if key in ints else np.float64))
    models = {int(sc.get("cloth_model", 0)) for sc in scenes if len(sc["tris"])}
    if len(models) > 1:
        raise ValueError("scenes of a batch must share the cloth model")
    out["cloth_model"] = models.pop() if models else 0
    out["n_scenes"] = len(scenes)
    out["scene_vert_offsets"] = np.cumsum([0] + [len(sc["rest_pos"]) for sc in scenes])
    out["bbox_diag"] = max(sc["bbox_diag"] for sc in scenes)
    out["newton_tol"] = float(newton_tol if newton_tol is not None else min(sc["newton_tol"] for sc in scenes))
    return out


def scene_by_name(name, **kw):
    return {"cubes": cubes_scene, "tori": tori_scene, "mixed": mixed_scene, "beam": beam_scene}[name](**kw)
