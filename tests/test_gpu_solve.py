"""GPU parity of the PEEC topology, the loop-space operator (eq. 8), the
diagonal-of-P preconditioner matrix (eq. 10) and the port R, L of a sweep
against the CPU oracle, through the C-ABI."""
import numpy as np
import pytest

import meshgen
from oracle import circuit
from oracle.esi import zs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import os

    import __graft_entry__
    import paper_2409_12375_gb300 as pkg
    if not os.path.exists(pkg.library_path()):
        __graft_entry__.build()
    return pkg


@pytest.fixture(scope="module")
def bar_ctx(lib, bar_mesh):
    x = lib.XRL.from_mesh(bar_mesh, fmm_order=8)
    yield x
    x.close()


@pytest.fixture(scope="module")
def coils_mesh_s():
    return meshgen.coils()


@pytest.fixture(scope="module")
def bar_circ(bar_mesh):
    return circuit.Circuit(bar_mesh)


def _loop_matrix(ctx, nbranch):
    ptr, col, val = ctx.export_loops()
    M = np.zeros((ptr.shape[0] - 1, nbranch))
    for l in range(ptr.shape[0] - 1):
        M[l, col[ptr[l]:ptr[l + 1]]] = val[ptr[l]:ptr[l + 1]]
    return M


def test_branches_match_oracle(bar_ctx, bar_circ):
    t, h = bar_ctx.export_branches()
    c = bar_circ
    assert t.shape[0] == c.n_branch
    live = c.live
    for b in range(c.n_cb):
        assert live[c.tail[b]] == t[b]
        if c.head[b] < c.n_live:
            assert live[c.head[b]] == h[b]
        else:
            assert h[b] == -1 - (c.head[b] - c.n_live)


def test_loops_are_a_cycle_basis(bar_ctx, bar_circ):
    M = _loop_matrix(bar_ctx, bar_circ.n_branch)
    assert M.shape[0] == bar_circ.M.shape[0]
    assert np.abs(M @ bar_circ.incidence().T).max() == 0.0
    assert np.linalg.matrix_rank(M) == M.shape[0]
    st = bar_ctx.stats()
    assert st["n_vertex_loops"] + st["n_global_loops"] == M.shape[0]


def _z_edge(c, f, P_full, diag_only=False):
    Pl = P_full[np.ix_(c.live, c.live)]
    if diag_only:
        Pl = np.diag(np.diag(Pl))
    d = c.zs_panels(f)
    core = np.diag(d) + 1j * 2 * np.pi * f * 1e-7 * Pl
    return sum(c.A[t] @ core @ c.A[t].T for t in range(3))


@pytest.mark.parametrize("f", [1e3, 1e9])
def test_operator_matches_oracle(bar_ctx, bar_circ, bar_dense_P, f):
    c = bar_circ
    M = _loop_matrix(bar_ctx, c.n_branch)[:, :c.n_cb]
    rng = np.random.default_rng(11)
    v = rng.standard_normal((2, M.shape[0])) + 1j * rng.standard_normal((2, M.shape[0]))
    w = bar_ctx.apply_operator(np.array([f, f]), v)
    Ze = _z_edge(c, f, bar_dense_P)
    ref = (M @ Ze @ M.T @ v.T).T
    err = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err


@pytest.mark.parametrize("nsys,p", [(8, 8), (16, 8), (16, 7)])
def test_double_float_operator_matches_fp64(lib, coils_mesh_s, nsys, p):
    """The mixed mode's FP64 residual operator against the plain FP64 kernels
    on the coils.  At 8 systems (48 columns) the near field and translations
    run in double-float on the FP32 pipes (~2^-44 per operation); at 16 (96
    columns) the M2L runs on the tensor cores in 5 integer slices of 7 bits
    (truncation ~2^-35 of max|M| max|T| per term), with 96-wide tiles at order
    8 and 64-wide ones at order 7.  Both evaluate the same FMM,
    so they agree far below the order-8 truncation (~1e-7) and the 1e-8
    residual target."""
    rng = np.random.default_rng(13)
    a = lib.XRL.from_mesh(coils_mesh_s, precision=0, fmm_order=p)
    b = lib.XRL.from_mesh(coils_mesh_s, precision=1, fmm_order=p)
    try:
        n = a.stats()["n_loops"]
        v = rng.standard_normal((nsys, n)) + 1j * rng.standard_normal((nsys, n))
        f = np.geomspace(1e3, 1e9, nsys)
        w0 = a.apply_operator(f, v)
        w1 = b.apply_operator(f, v)
    finally:
        a.close()
        b.close()
    err = np.linalg.norm(w1 - w0, axis=1) / np.linalg.norm(w0, axis=1)
    assert err.max() < 1e-10, err.max()


def test_precond_matrix_matches_oracle(bar_ctx, bar_circ, bar_dense_P):
    c = bar_circ
    M = _loop_matrix(bar_ctx, c.n_branch)[:, :c.n_cb]
    rng = np.random.default_rng(12)
    v = rng.standard_normal((2, M.shape[0])) + 1j * rng.standard_normal((2, M.shape[0]))
    f = np.array([1e5, 1e8])
    w = bar_ctx.apply_operator(f, v, precond_matrix=True)
    for s in range(2):
        Qe = _z_edge(c, f[s], bar_dense_P, diag_only=True)
        ref = M @ Qe @ M.T @ v[s]
        assert np.linalg.norm(w[s] - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("mesh_name", ["bar", "coils"])
def test_banded_precond_inverse(lib, bar_ctx, mesh_name):
    """Q(f)^-1 by the banded LDL^T + border factorisation, checked by
    applying Q (the sparse matrix of eq. 10) to the result."""
    ctx = bar_ctx
    if mesh_name == "coils":
        ctx = lib.XRL.from_mesh(meshgen.coils(), fmm_order=4)
    n = ctx.stats()["n_loops"]
    rng = np.random.default_rng(13)
    f = np.array([1e2, 1e6, 1e10])
    v = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    z = ctx.apply_operator(f, v, precond_inverse=True)
    back = ctx.apply_operator(f, z, precond_matrix=True)
    assert np.linalg.norm(back - v) / np.linalg.norm(v) < 1e-10
    if mesh_name == "coils":
        ctx.close()


def test_bar_sweep_matches_oracle(bar_ctx, bar_circ, bar_dense_P, bar_mesh):
    f = bar_mesh.freqs
    R, L = bar_ctx.solve(f)
    Ro, Lo, _ = bar_circ.solve(f, bar_dense_P)
    assert np.max(np.abs(R - Ro) / np.abs(Ro)) < 1e-4
    assert np.max(np.abs(L - Lo) / np.abs(Lo)) < 1e-4
    st = bar_ctx.stats()
    assert st["max_rel_res"] <= 1e-8


@pytest.mark.parametrize("p", [8, 7])
def test_mixed_precision_sweep_matches_oracle(lib, bar_circ, bar_dense_P, bar_mesh, p):
    """FP32 FMM inside FP64 FGMRES-IR, at order 8 and at the autotuned order
    7: the final FP64 residual still reaches 1e-8 and R, L match the oracle
    to 1e-4."""
    x = lib.XRL.from_mesh(bar_mesh, fmm_order=p, precision=1)
    f = bar_mesh.freqs
    R, L = x.solve(f)
    Ro, Lo, _ = bar_circ.solve(f, bar_dense_P)
    assert np.max(np.abs(R - Ro) / np.abs(Ro)) < 1e-4
    assert np.max(np.abs(L - Lo) / np.abs(Lo)) < 1e-4
    assert x.stats()["max_rel_res"] <= 1e-8
    x.close()


def test_bar_low_frequency_resistance(bar_ctx):
    R, L = bar_ctx.solve(np.array([1e-3]))
    rho_l_a = 10e-3 / (5.8e7 * 1e-6)
    assert abs(R[0, 0, 0] / rho_l_a - 1) < 1e-4


def test_two_bars_sweep(lib, two_bars_mesh, two_bars_dense_P):
    x = lib.XRL.from_mesh(two_bars_mesh, fmm_order=8)
    f = np.array([1e4, 1e9])
    R, L = x.solve(f)
    c = circuit.Circuit(two_bars_mesh)
    Ro, Lo, _ = c.solve(f, two_bars_dense_P)
    assert np.max(np.abs(R - Ro)) < 1e-4 * np.max(np.abs(Ro))
    assert np.max(np.abs(L - Lo)) < 1e-4 * np.max(np.abs(Lo))
    assert np.max(np.abs(L - np.transpose(L, (0, 2, 1)))) < 1e-6 * np.max(np.abs(L))
    x.close()


def test_error_codes(lib):
    from paper_2409_12375_gb300.xrl import XRLError
    m = meshgen.bar(length=2e-3, n_w=2, n_h=2, n_l=6)
    x = lib.XRL()
    with pytest.raises(XRLError) as e:
        x.solve(np.array([1e6]))
    assert e.value.code == 7           # XRL_ESTATE
    # open surface: drop one triangle
    x.set_mesh(m.xyz, m.tri[1:], m.cond[1:])
    with pytest.raises(XRLError) as e:
        x.setup()
    assert e.value.code == 2           # XRL_ETOPO
    x.set_mesh(m.xyz, m.tri, m.cond)
    with pytest.raises(XRLError) as e:
        x.add_port(np.array([0, 10 ** 6]), np.array([1]))
    assert e.value.code == 1           # XRL_EINVAL
    x.close()


@pytest.fixture(scope="module")
def bar_ctx_L(lib, bar_mesh):
    x = lib.XRL.from_mesh(bar_mesh, fmm_order=8, precond=3)
    yield x
    x.close()


def test_diag_L_precond_matrix_matches_oracle(bar_ctx_L, bar_circ, bar_dense_P):
    """The diagonal-of-L pencil (Sec. II-D, Table IV) against the oracle's
    Q_L in the library's own loop basis; its branch cross terms P_01 come
    from the rule-table kernel."""
    c = bar_circ
    M = _loop_matrix(bar_ctx_L, c.n_branch)
    rng = np.random.default_rng(21)
    v = rng.standard_normal((2, M.shape[0])) + 1j * rng.standard_normal((2, M.shape[0]))
    f = np.array([1e4, 1e9])
    w = bar_ctx_L.apply_operator(f, v, precond_matrix=True)
    for s in range(2):
        ref = circuit.precond_matrix_L(c, f[s], bar_dense_P, M=M) @ v[s]
        assert np.linalg.norm(w[s] - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("mesh_name", ["bar", "coils"])
def test_diag_L_banded_inverse(lib, bar_ctx_L, mesh_name):
    ctx = bar_ctx_L
    if mesh_name == "coils":
        ctx = lib.XRL.from_mesh(meshgen.coils(), fmm_order=4, precond=3)
    n = ctx.stats()["n_loops"]
    rng = np.random.default_rng(22)
    f = np.array([1e2, 1e6, 1e10])
    v = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    z = ctx.apply_operator(f, v, precond_inverse=True)
    back = ctx.apply_operator(f, z, precond_matrix=True)
    assert np.linalg.norm(back - v) / np.linalg.norm(v) < 1e-10
    if mesh_name == "coils":
        ctx.close()


def test_diag_L_sweep_matches_oracle(bar_ctx_L, bar_circ, bar_dense_P, bar_mesh):
    """The preconditioner changes the iterations, not the answer."""
    f = bar_mesh.freqs
    R, L = bar_ctx_L.solve(f)
    Ro, Lo, _ = bar_circ.solve(f, bar_dense_P)
    assert np.max(np.abs(R - Ro) / np.abs(Ro)) < 1e-4
    assert np.max(np.abs(L - Lo) / np.abs(Lo)) < 1e-4
    assert bar_ctx_L.stats()["max_rel_res"] <= 1e-8
