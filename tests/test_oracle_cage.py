"""Oracle pins of the cage parameterisation (Sec. "Caged Bunny"; CPU).

A surface vertex embedded in a hex cage sits at p = sum_k w_k c_k over the 8
corners of its cage cell (trilinear weights); its UNION Jacobian is w_k I3
over those 8 nodes, and a contact pair then couples the union of the nodes
of its vertices (compressed before the scatter).  Pinned here:
  * the position map against that definition, with random cage states;
  * the assembled gradient and exact Hessian of the caged blob in contact
    (with the ground and an affine box) against central differences of the
    oracle's energy;
  * the compressed sizes the paper prints for a point-point pair of caged
    vertices whose cells share 0, 1, 2, 4 or 8 cage vertices (48, 45, 42, 36,
    24), as the support of the assembled barrier Hessian.
"""
import json
import os

import numpy as np
import pytest

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_embedded_position_map_definition():
    s = scenes.caged_blob_scene(with_box=False)
    O = oracle.OracleSystem(s)
    x0, _ = O.initial_state()
    vnode, _, _ = O.vertex_info()
    rng = np.random.default_rng(8)
    x = x0 + 1e-3 * rng.normal(size=x0.shape)
    P = O.positions(x)
    cage_pos = lambda c: x[vnode[c]]
    for e, v in enumerate(s["embed_verts"]):
        want = sum(s["embed_w"][e][k] * cage_pos(s["embed_cage"][e][k]) for k in range(8))
        assert np.allclose(P[v], want, rtol=0, atol=1e-15)
    assert np.all(vnode[s["embed_verts"]] < 0) and O.nn == 4 * len(s["body_mass"]) + int((s["vert_body"] == -1).sum())


def _fd(f, x, h):
    out = []
    for i in range(x.size):
        e = np.zeros_like(x)
        e.flat[i] = h
        out.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack(out, axis=-1)


def test_caged_contact_derivatives_match_fd():
    s = scenes.caged_blob_scene(blob_h=0.02, cage_h=0.04)
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    rng = np.random.default_rng(9)
    x = x + 2e-5 * rng.normal(size=x.shape)
    pt, ee, pg = O.pairs(x)
    assert len(pg) > 0 and len(pt) + len(ee) > 0
    xt = O.xtilde(x, v)
    g = O.assemble(x, xt, project=False).ravel()
    gfd = _fd(lambda y: np.array(O.energy(y.reshape(-1, 3), xt)), x.ravel(), 1e-8)
    scale = np.abs(gfd).max()
    assert np.all(np.abs(g - gfd) <= 1e-6 * scale + 1e-5 * np.abs(gfd))
    O.assemble(x, xt, project=False)
    H = O.dense_hessian()
    Hfd = _fd(lambda y: O.assemble(y.reshape(-1, 3), xt, project=False).ravel(), x.ravel(), 1e-9)
    Hfd = 0.5 * (Hfd + Hfd.T)
    assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(Hfd).max()


def cage_pair_scene(shared, h=0.01, eps=2e-4):
    """A 4 x 3 x 3 cage with two small embedded triangles: one in cell (1, 1, 1)
    near a corner, one in the cell that shares `shared` corners with it (the
    same cell: 8, a face: 4, an edge: 2, a corner: 1, none: 0), placed so that
    their nearest vertices are within dhat.  Returns the scene and the DOF
    state (for `0` the far cell's nodes are translated next to the first)."""
    cell_b = {8: (1, 1, 1), 4: (2, 1, 1), 2: (2, 2, 1), 1: (2, 2, 2), 0: (3, 1, 1)}[shared]
    dims = (4, 3, 3)
    parts = scenes._empty_parts()
    cv = scenes.hex_grid(*dims, h)
    coff = scenes._add_soft(parts, cv, scenes.kuhn_tets(*dims), 3e4, 0.3, 1000.0, surface=False)
    corner = np.array([2.0, 2.0, 2.0]) * h  # the far corner of cell (1, 1, 1)
    qa = corner - np.array([eps, eps, eps])
    d = 0.2 * h
    if shared == 8:  # below the first triangle's plane, in the same cell
        pa = qa - np.array([0.0, 0.0, 2.5 * eps])
        a1, a2 = np.array([0.0, 0.0, -d]), np.array([-d, 0.0, -d])
    else:
        sg = np.array([1.0, 1.0, 1.0])
        if shared == 0:
            pa = np.array([3.0, 1.0, 1.0]) * h + 3 * eps  # inside cell (3, 1, 1), moved later
        else:
            sg = np.array([1.0 if c > 1 else -1.0 for c in cell_b])
            pa = corner + sg * eps
        a1, a2 = np.array([d * sg[0], 0.0, 0.0]), np.array([0.0, 0.0, d * sg[2]])
    tri_q = np.array([qa, qa - [d, 0, 0], qa - [0, d, 0]])
    tri_p = np.array([pa, pa + a1, pa + a2])
    verts = np.concatenate([tri_q, tri_p])
    scenes._add_embedded_surface(parts, verts, np.array([[0, 2, 1], [3, 4, 5]]), coff, np.zeros(3), h, dims)
    s = scenes.finalize_scene(parts, "cage_pair", 0.01, 1e-3, 1e4, 1, planes=np.zeros((0, 4)))
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    if shared == 0:
        # move cell (3, 1, 1) rigidly so that its triangle's first vertex lands
        # 0.35 mm from the other triangle's nearest vertex
        vid = lambda i, j, k: i + (dims[0] + 1) * (j + (dims[1] + 1) * k)
        cell = [vid(3 + a, 1 + b, 1 + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
        vnode, _, _ = O.vertex_info()
        shift = (qa + np.array([3.5e-4, 0.0, 0.0])) - pa
        for c in cell:
            x[vnode[coff + c]] += shift
    return s, O, x, v


def test_compressed_sizes_of_caged_point_point_pairs():
    sizes = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["caged_pp_compressed"]
    for shared in (8, 4, 2, 1, 0):
        s, O, x, v = cage_pair_scene(shared)
        pt, ee, pg = O.pairs(x)
        assert len(pt) + len(ee) > 0, shared
        xt = O.xtilde(x, v)
        O0 = oracle.OracleSystem(s, kappa=0.0)
        O.assemble(x, xt, project=False)
        H1 = O.dense_hessian()
        O0.assemble(x, xt, project=False)
        H0 = O0.dense_hessian()
        support = np.nonzero(np.abs(H1 - H0).sum(0) > 0)[0]
        assert len(support) == sizes[str(shared)], (shared, len(support))
