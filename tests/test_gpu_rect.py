"""GPU parity on hybrid triangle/rectangle meshes (Sec. II-A, Figs. 1-2)
against the oracle, through the C-ABI: the octree (bit-exact), the rule-table
P entries of rectangles (direct sum), the FMM products in both precisions,
the loop operator and the preconditioner pencil, and the port R, L."""
import numpy as np
import pytest

import meshgen
from oracle import circuit, panels, tree

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-6


@pytest.fixture(scope="module")
def lib():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


def _hyb_coil():
    return meshgen.coils(outer=2e-3, turns=1, n_w=2, step=0.2e-3, n_coils=1, rect=True,
                         n_freq=4, fmin=1e3, fmax=1e9)


def _rect_bar():
    return meshgen.bar(jitter=0.0, rect=True, n_l=20, freqs=(1e-3, 1e5, 1e9))


@pytest.fixture(scope="module", params=["hybrid_coil", "rect_bar"])
def case(request, lib):
    m = _hyb_coil() if request.param == "hybrid_coil" else _rect_bar()
    circ = circuit.Circuit(m)
    P = panels.dense_P_panels(circ.geom)
    ctx = lib.XRL.from_mesh(m, fmm_order=8)
    yield m, circ, P, ctx
    ctx.close()


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


def _check_tree(ctx, mesh):
    if ctx.opts.mac_theta > 0:
        ref = tree.build_mac(mesh.xyz, mesh.tri, leaf_target=ctx.opts.leaf_target, theta=ctx.opts.mac_theta,
                             cap=0.0)
    else:
        ref = tree.build(mesh.xyz, mesh.tri, leaf_target=ctx.opts.leaf_target, ws=ctx.opts.separation)
    keys, perm, leaf = ctx.export_tree()
    assert np.array_equal(keys, ref["keys"])
    assert np.array_equal(perm, ref["perm"])
    assert np.array_equal(leaf, ref["leaf_of"])
    assert ctx.stats()["n_levels"] == ref["L"] + 1


def test_hybrid_tree_bit_exact(case):
    m, _, _, ctx = case
    _check_tree(ctx, m)


def test_hybrid_direct_sum_matches_oracle(case):
    import torch
    _, _, P, ctx = case
    rng = np.random.default_rng(31)
    x = rng.standard_normal((3, P.shape[0]))
    xd = _dev(x)
    yd = torch.empty_like(xd)
    ctx.direct_mvm_device(xd, yd)
    torch.cuda.synchronize()
    ref = x @ P.T
    y = yd.cpu().numpy()
    assert np.max(np.abs(y - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("nc", [1, 6, 64])
def test_hybrid_fmm_matches_oracle(case, nc):
    import torch
    _, _, P, ctx = case
    rng = np.random.default_rng(40 + nc)
    x = rng.standard_normal((nc, P.shape[0]))
    ref = x @ P.T
    y = ctx.fmm_mvm(x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-6
    x32 = x.astype(np.float32)
    xd = torch.tensor(x32, device="cuda:0")
    yd = torch.empty_like(xd)
    ctx.fmm_mvm32_device(xd, yd)
    torch.cuda.synchronize()
    ref32 = x32.astype(np.float64) @ P.T
    y32 = yd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(y32 - ref32) / np.linalg.norm(ref32) < FP32_TOL


def _loop_matrix(ctx, nbranch):
    ptr, col, val = ctx.export_loops()
    M = np.zeros((ptr.shape[0] - 1, nbranch))
    for l in range(ptr.shape[0] - 1):
        M[l, col[ptr[l]:ptr[l + 1]]] = val[ptr[l]:ptr[l + 1]]
    return M


def test_hybrid_operator_and_precond_match_oracle(case):
    _, c, P, ctx = case
    M = _loop_matrix(ctx, c.n_branch)
    n = M.shape[0]
    rng = np.random.default_rng(32)
    v = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    f = np.array([1e4, 1e9])
    w = ctx.apply_operator(f, v)
    q = ctx.apply_operator(f, v, precond_matrix=True)
    Pl = P[np.ix_(c.live, c.live)]
    Mc = M[:, :c.n_cb]
    for s in range(2):
        d = c.zs_panels(f[s])
        Ze = sum(c.A[t] @ (np.diag(d) + 1j * 2 * np.pi * f[s] * 1e-7 * Pl) @ c.A[t].T for t in range(3))
        ref = Mc @ Ze @ Mc.T @ v[s]
        assert np.linalg.norm(w[s] - ref) / np.linalg.norm(ref) < 1e-6
        refq = circuit.precond_matrix(c, f[s], P, M=M) @ v[s]
        assert np.linalg.norm(q[s] - refq) / np.linalg.norm(refq) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_hybrid_sweep_matches_oracle(lib, case, precision):
    m, c, P, _ = case
    x = lib.XRL.from_mesh(m, fmm_order=8, precision=precision)
    try:
        R, L = x.solve(m.freqs)
        assert x.stats()["max_rel_res"] <= 1e-8
    finally:
        x.close()
    Ro, Lo, _ = c.solve(m.freqs, P)
    assert np.max(np.abs(R - Ro) / np.abs(Ro)) < 1e-4
    assert np.max(np.abs(L - Lo) / np.abs(Lo)) < 1e-4
    if m.name == "bar":
        # DC limit of the rectangle-meshed bar: rho l / A (ESI thickness 2A/perimeter)
        assert abs(R[0, 0, 0] / (10e-3 / (5.8e7 * 1e-6)) - 1) < 1e-4


def test_full_size_hybrid_coils_sampled_rows(lib):
    """The coils meshed with rectangles on the straight runs and triangles at
    the mitred corners (12,756 panels): the octree bit for bit and sampled
    oracle rows of P times x at 6 columns."""
    m = meshgen.coils(rect=True)
    x = lib.XRL.from_mesh(m, fmm_order=8)
    try:
        _check_tree(x, m)
        rng = np.random.default_rng(33)
        N = m.n_tri
        v = rng.standard_normal((6, N))
        y = x.fmm_mvm(v)
    finally:
        x.close()
    rows = rng.choice(N, 12, replace=False)
    Pr = panels.rows_P_panels(panels.Panels(m.xyz, m.tri), rows)
    ref = v @ Pr.T
    err = np.linalg.norm(y[:, rows] - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err


def test_hybrid_mesh_argument_errors(lib):
    """xrl_set_mesh_panels: a 4-vertex panel that is not a parallelogram is
    XRL_EINVAL, a repeated vertex in a panel XRL_ETOPO, and a 4th slot below -1
    XRL_EINVAL; the context stays usable for a valid mesh afterwards."""
    m = _rect_bar()
    x = lib.XRL()
    try:
        bad = np.asarray(m.xyz).copy()
        q = int(np.flatnonzero(m.tri[:, 3] >= 0)[0])
        bad[m.tri[q, 2]] += np.array([1e-5, 2e-5, 0.0])
        with pytest.raises(lib.XRLError) as e:
            x.set_mesh(bad, m.tri, m.cond)
        assert e.value.code == 1
        rep = m.tri.copy()
        rep[q, 1] = rep[q, 0]
        with pytest.raises(lib.XRLError) as e:
            x.set_mesh(m.xyz, rep, m.cond)
        assert e.value.code == 2
        neg = m.tri.copy()
        neg[q, 3] = -2
        with pytest.raises(lib.XRLError) as e:
            x.set_mesh(m.xyz, neg, m.cond)
        assert e.value.code == 1
        x.set_mesh(m.xyz, m.tri, m.cond)
        x.set_conductors(m.sigma, m.thickness)
        term = np.asarray(m.term)
        for s_, k in m.ports:
            x.add_port(np.flatnonzero(term == s_), np.flatnonzero(term == k))
        x.setup()
        assert x.stats()["n_panels"] == m.n_tri
    finally:
        x.close()
    with pytest.raises(lib.XRLError) as e:
        lib.XRL(precond=5)
    assert e.value.code == 1


def test_full_size_hybrid_coils_fp32_tensor_core_product(lib):
    """The FP32 product of the full hybrid coils at 384 columns (every leaf has
    at most 64 padded panels, so every sibling pair shares a CTA in the near
    field and the M2L): against the FP64 product, column by column, with the
    bound of the triangle coils' test."""
    import torch
    m = meshgen.coils(rect=True)
    x = lib.XRL.from_mesh(m, fmm_order=7)
    try:
        rng = np.random.default_rng(34)
        v = rng.standard_normal((384, m.n_tri)).astype(np.float32)
        y64 = x.fmm_mvm(v.astype(np.float64))
        xd = torch.tensor(v, device="cuda:0")
        yd = torch.empty_like(xd)
        x.fmm_mvm32_device(xd, yd)
        torch.cuda.synchronize()
        y32 = yd.cpu().numpy().astype(np.float64)
    finally:
        x.close()
    e = (np.linalg.norm(y32 - y64, axis=1) / np.linalg.norm(y64, axis=1)).max()
    assert e < 2e-5, e
