"""The nested-dissection plan of the interface system (host only, no GPU).

``hps_interface_plan`` returns the merge tree that the GPU factorisation
follows.  Here the tree is checked for structure (every shared face is
eliminated by exactly one merge, the root keeps no boundary) and then used
in a plain numpy elimination of the oracle's leaf DtN maps: the face values
it gives must equal the oracle's two-level solve with the host sparse LU
(Sec. 3.1 assembly), for uneven grids, variable b and nonzero Dirichlet data.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle import global_solve as gs


@pytest.fixture(scope="module")
def H():
    import paper_2503_04033_gb300 as H
    if not os.path.exists(H.library_path()):
        from paper_2503_04033_gb300 import build
        build.build()
    H.load_library()
    return H


def _split(row, lists):
    a, b, _, _, na1, nsep, nb2, off = (int(v) for v in row)
    a1 = lists[off:off + na1]
    a3 = lists[off + na1:off + na1 + nsep]
    b2 = lists[off + na1 + nsep:off + na1 + nsep + nb2]
    b3 = lists[off + na1 + nsep + nb2:off + na1 + 2 * nsep + nb2]
    return a, b, a1, a3, b2, b3


def _pos(slots, qq):
    if len(slots) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.concatenate([np.arange(s * qq, (s + 1) * qq) for s in slots])


def merge_solve(nodes, lists, nbox, qq, T, h):
    """Face values [nbox, m] at the shared faces (outer faces left 0) by the
    plan's eliminations: the upward pass forms each merge's map and flux, the
    downward pass the separator values."""
    Tm = {bx: T[bx] for bx in range(nbox)}
    hm = {bx: h[bx] for bx in range(nbox)}
    saved = []
    for r, row in enumerate(nodes):
        a, b, a1, a3, b2, b3 = _split(row, lists)
        p1, p3a, p2, p3b = _pos(a1, qq), _pos(a3, qq), _pos(b2, qq), _pos(b3, qq)
        W = Tm[a][np.ix_(p3a, p3a)] + Tm[b][np.ix_(p3b, p3b)]
        S = -np.linalg.solve(W, np.hstack([Tm[a][np.ix_(p3a, p1)], Tm[b][np.ix_(p3b, p2)]]))
        E = np.vstack([Tm[a][np.ix_(p1, p3a)], Tm[b][np.ix_(p2, p3b)]])
        e1, e2 = len(p1), len(p2)
        Tn = np.zeros((e1 + e2, e1 + e2))
        Tn[:e1, :e1] = Tm[a][np.ix_(p1, p1)]
        Tn[e1:, e1:] = Tm[b][np.ix_(p2, p2)]
        Tn += E @ S
        y = np.linalg.solve(W, hm[a][p3a] + hm[b][p3b])
        Tm[nbox + r] = Tn
        hm[nbox + r] = np.concatenate([hm[a][p1], hm[b][p2]]) - E @ y
        saved.append((a, b, p1, p3a, p2, p3b, S, y))
    m = T.shape[1]
    u = {}
    if len(nodes):
        u[nbox + len(nodes) - 1] = np.zeros(0)
    ub = np.zeros((nbox, m))
    for r in range(len(nodes) - 1, -1, -1):
        a, b, p1, p3a, p2, p3b, S, y = saved[r]
        uX = u[nbox + r]
        u3 = S @ uX - y
        for child, pe, p3, part in ((a, p1, p3a, uX[:len(p1)]), (b, p2, p3b, uX[len(p1):])):
            vec = ub[child] if child < nbox else np.zeros(len(hm[child]))
            vec[pe] = part
            vec[p3] = u3
            if child >= nbox:
                u[child] = vec
    return ub


@pytest.mark.parametrize("nb", [(2, 2, 2), (3, 1, 2), (4, 2, 1), (1, 1, 3), (3, 3, 2)])
def test_plan_structure(H, nb):
    p = 6
    q = p - 2
    nodes, lists = H.hps_interface_plan(p, nb)
    grid = gs.InterfaceGrid(p, nb)
    nbox = grid.nbox
    assert len(nodes) == nbox - 1
    # every shared face is eliminated exactly once
    assert int(nodes[:, 5].sum()) == grid.n_iface_faces if nbox > 1 else len(nodes) == 0
    if nbox > 1:
        root = nodes[-1]
        assert root[4] == 0 and root[6] == 0
        assert list(nodes[:, 2]) == sorted(nodes[:, 2])
        children = sorted(int(c) for c in nodes[:, :2].reshape(-1))
        assert children == list(range(2 * nbox - 2))
    assert q > 0


@pytest.mark.parametrize("nb,kappa", [((2, 2, 2), 0.0), ((3, 1, 2), 4.0), ((3, 2, 2), 2.5), ((1, 2, 1), 3.0)])
def test_plan_elimination_matches_sparse_lu(H, nb, kappa):
    """Plan + numpy elimination of the oracle's maps = the oracle's sparse LU
    solve, with variable b, a body load and nonzero Dirichlet data."""
    p = 5
    q = p - 2
    qq = q * q
    grid = gs.InterfaceGrid(p, nb, L=(1.0, 0.8, 1.2))
    nbox = grid.nbox
    n, m = oracle.sizes(p)
    rng = np.random.default_rng(11)
    xyz = [oracle.node_coords(p, grid.box_lo(bx), grid.h) for bx in range(nbox)]
    b = [1.0 + 0.3 * np.sin(2 * x[:, 0] + x[:, 1] - x[:, 2]) for x in xyz]
    f = [np.cos(x[:, 0] + 2 * x[:, 2]) for x in xyz]
    g_dir = rng.standard_normal(grid.n_dir)
    ref = gs.hps_solve_boxes(grid, kappa, b, f, g_dir)
    T = np.empty((nbox, m, m))
    h = np.empty((nbox, m))
    for bx in range(nbox):
        T[bx], _, info = oracle.leaf_dtn(p, grid.h, kappa, b[bx], want_S=False)
        assert info == 0
        _, hf, info = oracle.leaf_particular(p, grid.h, kappa, b[bx], f[bx][None, :])
        assert info == 0
        isi, gid = grid.local_to_global(bx)
        rd = np.nonzero(~isi)[0]
        h[bx] = hf[0] + T[bx][:, rd] @ g_dir[gid[rd]]
    nodes, lists = H.hps_interface_plan(p, nb)
    ub = merge_solve(nodes, lists, nbox, qq, T, h)
    scale = np.abs(ref["u_iface"]).max()
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        np.testing.assert_allclose(ub[bx, isi], ref["u_iface"][gid[isi]], rtol=0, atol=1e-11 * scale)


def test_plan_rejects_bad_arguments(H):
    with pytest.raises(H.HpsError):
        H.hps_interface_plan(2, (2, 2, 2))
    with pytest.raises(H.HpsError):
        H.hps_interface_plan(8, (0, 1, 1))


@pytest.mark.parametrize("nb,kappa", [((2, 2), 0.0), ((3, 2), 4.0), ((4, 3), 2.0), ((1, 3), 3.0)])
def test_plan_2d_elimination_matches_sparse_lu(H, nb, kappa):
    """The 2-D plan (edges of q nodes as the slots): a numpy elimination that
    follows it on the oracle's 2-D leaf maps equals the oracle's two-level
    solve with the host sparse LU."""
    from oracle import global_solve_2d as g2
    p = 6
    q = p - 2
    grid = g2.InterfaceGrid2D(p, nb, lo=(0.2, -0.1), L=(1.1, 0.9))
    nbox = grid.nbox
    n, m = oracle.sizes_2d(p)
    rng = np.random.default_rng(5)
    xy = [oracle.node_coords_2d(p, grid.box_lo(bx), grid.h) for bx in range(nbox)]
    b = [1.0 + 0.3 * np.sin(2 * x[:, 0] - x[:, 1]) for x in xy]
    f = [np.cos(x[:, 0] + 2 * x[:, 1]) for x in xy]
    g_dir = rng.standard_normal(grid.n_dir)
    ref = g2.hps_solve_2d(grid, kappa, b, f, g_dir)
    T = np.empty((nbox, m, m))
    h = np.empty((nbox, m))
    for bx in range(nbox):
        T[bx], _, info = oracle.leaf_dtn_2d(p, grid.h, kappa, b[bx], want_S=False)
        assert info == 0
        _, hf, _ = oracle.leaf_particular_2d(p, grid.h, kappa, b[bx], f[bx][None, :])
        isi, gid = grid.local_to_global(bx)
        rd = np.nonzero(~isi)[0]
        h[bx] = hf[0] + T[bx][:, rd] @ g_dir[gid[rd]]
    nodes, lists = H.hps_interface2d_plan(p, nb)
    assert len(nodes) == nbox - 1
    if nbox > 1:
        assert int(nodes[:, 5].sum()) * q == grid.n_iface
    ub = merge_solve(nodes, lists, nbox, q, T, h)
    scale = np.abs(ref["u_iface"]).max()
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        np.testing.assert_allclose(ub[bx, isi], ref["u_iface"][gid[isi]], rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("nb,top,levels", [((4, 4, 4), 16, 6), ((8, 8, 8), 64, 9), ((8, 4, 2), 8, 6)])
def test_plan_sizes_of_uniform_grids(H, nb, top, levels):
    """Nested dissection of a uniform grid: the root's separator is the
    mid-plane across the longest axis (top faces), the tree has
    ceil(log2) levels per axis, and each level's separators together hold
    one plane of faces per split."""
    nodes, lists = H.hps_interface_plan(6, nb)
    grid = gs.InterfaceGrid(6, nb)
    assert len(nodes) == grid.nbox - 1
    assert int(nodes[-1, 5]) == top and nodes[-1, 4] == 0 and nodes[-1, 6] == 0
    assert int(nodes[:, 2].max()) == levels
    assert int(nodes[:, 5].sum()) == grid.n_iface_faces
    # children come from lower levels
    for row in nodes:
        for c in row[:2]:
            if c >= grid.nbox:
                assert nodes[c - grid.nbox, 2] < row[2]
