"""Pins of the 2D 9-point oracle (Sec. IV-A, "SpMV (2D)") against closed
forms, dense assembly, an independent column (scatter) formulation, direct
solves and tridiagonal reductions (CPU only).  ``test_planted_*`` plant
mistakes in the oracle and check that a pin catches them."""

import numpy as np
import pytest

import synth
from oracle import bicgstab as ob
from oracle import counts, direct, stencil9
from tests.conftest import golden

# (dx, dy) of each direction, written out here rather than taken from the
# oracle so that a wrong offset table in the oracle is caught
OFFSETS = {"xm": (-1, 0), "xp": (1, 0), "ym": (0, -1), "yp": (0, 1),
           "xmym": (-1, -1), "xpym": (1, -1), "xmyp": (-1, 1), "xpyp": (1, 1)}
# distinct constant coefficients: a swapped pair of directions changes A u
CONST = {"diag": 9.5, "xm": -1.3, "xp": -0.7, "ym": -1.1, "yp": -0.9,
         "xmym": -0.21, "xpym": -0.43, "xmyp": -0.37, "xpyp": -0.55}


def rand9(nx, ny, seed):
    p = synth.varcoef9(nx, ny, seed=seed, dtype=np.float64)
    return dict(p.coef), p.b.astype(np.float64)


def quadratic_check9(nx, ny, coef):
    """Max relative deviation of A u from the closed form on interior cells.

    For u = q0 + q1 x + q2 y + q3 x^2 + q4 x y + q5 y^2 the shift by (dx, dy)
    is exactly u + dx u_x + dy u_y + q3 dx^2 + q4 dx dy + q5 dy^2, so for
    constant coefficients A u = d u + sum_e c_e u(x + dx_e, y + dy_e) has a
    closed form.
    """
    rng = np.random.default_rng(11)
    q = rng.uniform(-1, 1, 6)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    u = q[0] + q[1] * x + q[2] * y + q[3] * x * x + q[4] * x * y + q[5] * y * y
    ux = q[1] + 2 * q[3] * x + q[4] * y
    uy = q[2] + q[4] * x + 2 * q[5] * y
    expect = coef["diag"] * u
    for name, (dx, dy) in OFFSETS.items():
        shift = u + dx * ux + dy * uy + q[3] * dx * dx + q[4] * dx * dy + q[5] * dy * dy
        expect = expect + coef[name] * shift
    got = stencil9.apply(nx, ny, coef, u.reshape(-1)).reshape(ny, nx)
    inner = (slice(1, -1), slice(1, -1))
    return np.max(np.abs(got[inner] - expect[inner]) / (1 + np.abs(expect[inner])))


def test_9pt_exact_on_quadratics():
    assert quadratic_check9(11, 9, CONST) < 1e-13


@pytest.mark.parametrize("swap", [("xpym", "xmyp"), ("xm", "ym"), ("xmym", "xpyp")])
def test_planted_wrong_offset_is_caught(monkeypatch, swap):
    bad = dict(stencil9.OFFS)
    a, b = swap
    bad[a], bad[b] = bad[b], bad[a]
    monkeypatch.setattr(stencil9, "OFFS", bad)
    assert quadratic_check9(11, 9, CONST) > 1e-3


def test_planted_dropped_corner_is_caught(monkeypatch):
    monkeypatch.setattr(stencil9, "DIRS", stencil9.DIRS[:-1])
    assert quadratic_check9(11, 9, CONST) > 1e-3


@pytest.mark.parametrize("jk", [(1, 1), (2, 3), (5, 1), (7, 6)])
def test_9pt_tensor_product_eigenpairs(jk):
    nx, ny = 12, 9
    a0, ax, ay, c = 8.0, -1.2, -0.8, -0.5
    coef = {"diag": a0, "xm": ax, "xp": ax, "ym": ay, "yp": ay,
            "xmym": c, "xpym": c, "xmyp": c, "xpyp": c}
    lam, v = direct.ninepoint_eigenpair(nx, ny, a0, ax, ay, c, *jk)
    assert np.max(np.abs(stencil9.apply(nx, ny, coef, v) - lam * v)) < 1e-13


def test_9pt_spectrum_of_dense_matrix():
    # the full spectrum of the assembled matrix is the closed-form set
    nx, ny = 6, 5
    a0, ax, ay, c = 8.0, -1.0, -1.0, -1.0     # the "Mehrstellen" 9-point Laplacian
    coef = {"diag": a0, "xm": ax, "xp": ax, "ym": ay, "yp": ay,
            "xmym": c, "xpym": c, "xmyp": c, "xpyp": c}
    ev = np.sort(np.linalg.eigvalsh(stencil9.assemble_dense(nx, ny, coef)))
    want = np.sort([direct.ninepoint_eigenpair(nx, ny, a0, ax, ay, c, j, k)[0]
                    for j in range(1, nx + 1) for k in range(1, ny + 1)])
    assert np.max(np.abs(ev - want)) < 1e-12


def test_9pt_dense_assembly_matches_apply():
    nx, ny = 7, 6
    coef, _ = rand9(nx, ny, 3)
    v = np.random.default_rng(1).standard_normal(nx * ny)
    a = stencil9.assemble_dense(nx, ny, coef)
    assert np.max(np.abs(a @ v - stencil9.apply(nx, ny, coef, v))) < 1e-13
    # each row has at most 9 entries, at the stencil's offsets
    assert np.count_nonzero(a[nx + 1]) == 9            # an interior row
    assert np.count_nonzero(a[0]) == 4                 # a corner row


def test_9pt_transpose():
    nx, ny = 7, 5
    coef, _ = rand9(nx, ny, 4)
    t = stencil9.transpose_coef(nx, ny, coef)
    a = stencil9.assemble_dense(nx, ny, coef)
    assert np.array_equal(stencil9.assemble_dense(nx, ny, t), a.T)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(nx * ny), rng.standard_normal(nx * ny)
    lhs = stencil9.apply(nx, ny, coef, x) @ y
    rhs = x @ stencil9.apply(nx, ny, t, y)
    assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


def test_9pt_column_formulation_matches_rows():
    """The paper's formulation (each cell scatters its column's products
    into its neighbours' outputs) equals the row (gather) form, and the
    column arrays hold exactly the dense matrix's column entries."""
    nx, ny = 9, 8
    coef, _ = rand9(nx, ny, 5)
    cols = stencil9.rows_to_columns(nx, ny, coef)
    v = np.random.default_rng(3).standard_normal(nx * ny)
    y_rows = stencil9.apply(nx, ny, coef, v)
    y_cols = stencil9.apply_columns(nx, ny, cols, v)
    assert np.max(np.abs(y_rows - y_cols)) < 1e-13 * np.max(np.abs(y_rows))
    a = stencil9.assemble_dense(nx, ny, coef)
    for name, (dx, dy) in OFFSETS.items():
        for j in range(nx * ny):
            x, y = j % nx, j // nx
            if 0 <= x + dx < nx and 0 <= y + dy < ny:
                assert cols[name][j] == a[j + dx + nx * dy, j]
            else:
                assert cols[name][j] == 0.0


def test_9pt_jacobi_scaling_is_row_scaling():
    nx, ny = 6, 7
    coef, b = rand9(nx, ny, 6)
    a = stencil9.assemble_dense(nx, ny, coef)
    d = np.diag(a).copy()
    scaled = stencil9.jacobi_scale(nx, ny, coef, "f64")
    assert np.allclose(stencil9.assemble_dense(nx, ny, scaled), a / d[:, None], rtol=0,
                       atol=1e-16)
    s32 = stencil9.jacobi_scale(nx, ny, coef, "f32")
    for k in s32:
        assert np.array_equal(s32[k], s32[k].astype(np.float32).astype(np.float64))
    assert np.allclose(stencil9.scale_rhs(nx, ny, coef, b), b / d)


def test_bicgstab9_matches_direct_solve():
    nx, ny = 11, 9
    coef, b = rand9(nx, ny, 7)
    xd = direct.dense_solve9(nx, ny, coef, b)
    r = ob.bicgstab9(nx, ny, coef, b, tol=1e-13, maxit=500)
    assert r.status == ob.OK
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-11
    assert r.true_resid_orig < 1e-12
    # and from a nonzero start, without Jacobi scaling
    x0 = np.random.default_rng(4).standard_normal(nx * ny)
    r = ob.bicgstab9(nx, ny, coef, b, x0=x0, tol=1e-13, maxit=500, jacobi=False)
    assert r.status == ob.OK
    assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-11


@pytest.mark.parametrize("shape", [(40, 1), (1, 40)])
def test_bicgstab9_single_row_or_column_is_tridiagonal(shape):
    # with one row (column) every neighbour but the two along x (y) is
    # off-mesh: the system is tridiagonal and the Thomas algorithm solves it
    nx, ny = shape
    coef, b = rand9(nx, ny, 8)
    lo, hi = ("xm", "xp") if ny == 1 else ("ym", "yp")
    xt = direct.thomas(coef[lo], coef["diag"], coef[hi], b)
    r = ob.bicgstab9(nx, ny, coef, b, tol=1e-14, maxit=200)
    assert r.status == ob.OK
    assert np.linalg.norm(r.x - xt) / np.linalg.norm(xt) < 1e-12


def test_bicgstab9_merged_tracks_algorithm_1():
    nx, ny = 14, 10
    coef, b = rand9(nx, ny, 9)
    a = ob.bicgstab9(nx, ny, coef, b, tol=1e-12, maxit=500)
    m = ob.bicgstab9_merged(nx, ny, coef, b, tol=1e-12, maxit=500)
    k = min(len(a.hist), len(m.hist), 10)
    assert np.max(np.abs(a.hist[:k] - m.hist[:k]) / a.hist[:k]) < 1e-9
    xd = direct.dense_solve9(nx, ny, coef, b)
    assert m.status == ob.OK
    assert np.linalg.norm(m.x - xd) / np.linalg.norm(xd) < 1e-10


def test_bicgstab9_history_tracks_true_residual():
    nx, ny = 30, 25
    coef, b = rand9(nx, ny, 10)
    r = ob.bicgstab9(nx, ny, coef, b, tol=1e-10, maxit=500)
    assert r.status == ob.OK and r.hist[-1] <= 1e-10
    assert r.true_resid < 2e-10


def test_paper_2d_numbers():
    g = {row[0]: float(row[1]) for row in golden("paper_numbers.txt")}
    # both 2D geometries are one sub-block per core over the same fabric edge
    edge = g["mesh2d_max"] / g["block2d_max"]
    assert edge == g["mesh2d_small"] / g["block2d_small"] == g["mesh_x"]
    assert counts.matvec_ops_9pt() == g["flops_9pt_matvec"]
    assert counts.matvec_ops_9pt(with_diagonal=False) == 16
    assert counts.ops_per_point_9pt() == 52
    assert counts.bytes_per_cell_9pt(4, 4, 4) == 132
    assert counts.bytes_per_cell_9pt(2, 2, 4) == 70


def test_synth9_dominance_and_sampling():
    nx, ny = 37, 21
    p = synth.varcoef9(nx, ny, seed=12)
    off = sum(np.abs(p.coef[d].astype(np.float64)) for d in synth.DIRS9)
    margin = p.coef["diag"].astype(np.float64) - off
    assert margin.min() > 0.009 and margin.max() < 0.1001
    for d in synth.DIRS9:
        assert -1.5 <= p.coef[d].min() and p.coef[d].max() <= -0.5
    idx = np.array([0, 1, nx, nx * ny - 1, 400])
    c, b = synth.varcoef9_at(nx, ny, idx, seed=12)
    for k in c:
        assert np.array_equal(c[k], p.coef[k][idx])
    assert np.array_equal(b, p.b[idx])
