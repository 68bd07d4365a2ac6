"""Operation and byte counts per mesh point per BiCGStab iteration.

Test infrastructure only.

Table I of the paper counts, per mesh point and iteration, the operations of
two matrix-vector products, four inner products and six AXPYs.  Its
single-precision columns are 22 additions and 22 multiplications (44 in
all); its mixed columns are 18 half-precision additions, 22 half-precision
multiplications and 4 single-precision additions (also 44).  Sec. V turns 44
operations per point into the reported rate (0.86 PFLOPS at 28.1 us per
iteration on the 600 x 595 x 1536 mesh).

``bytes_per_cell`` is this project's memory-traffic model of one iteration of
the fused three-kernel schedule: 12 coefficient words (6 per stencil sweep),
15 Krylov-vector words and 2 iterate words.
"""

# (additions, multiplications) per point per iteration, by operation class
TABLE_I_SINGLE = {"matvec": (12, 12), "dot": (4, 4), "axpy": (6, 6)}
# (half adds, half mults, single adds)
TABLE_I_MIXED = {"matvec": (12, 12, 0), "dot": (0, 4, 4), "axpy": (6, 6, 0)}


def ops_per_point():
    """Total operations per mesh point per iteration from Table I."""
    single = sum(a + m for a, m in TABLE_I_SINGLE.values())
    mixed = sum(sum(v) for v in TABLE_I_MIXED.values())
    return single, mixed


def ops_from_algorithm():
    """Table I derived from Algorithm 1's structure.

    Each of the two matvecs with a unit diagonal does 6 multiplications and 6
    additions per point; each of the four inner products one multiply and one
    add; each of the six AXPY-type updates (``q``, the two ``x`` terms, ``r``,
    and the two in ``p``) one multiply and one add.
    """
    matvec = 2 * 6
    dots = 4
    axpys = 6
    return {"matvec": (matvec, matvec), "dot": (dots, dots), "axpy": (axpys, axpys)}


def pflops(nx, ny, nz, seconds_per_iter, ops=44):
    return ops * nx * ny * nz / seconds_per_iter / 1e15


def bytes_per_cell(w_coef, w_vec, w_x):
    """Fused-schedule HBM bytes per cell per iteration: 12 w_c + 15 w_v + 2 w_x."""
    return 12 * w_coef + 15 * w_vec + 2 * w_x


def paper_storage_words(z):
    """Per-core storage of Sec. IV: six diagonals and four vectors of length
    Z (q and r_{i+1} reuse the storage of s and y), 10 Z words."""
    return 10 * z


def ops_per_point_9pt():
    """Credited operations per point per BiCGStab iteration on the 2D 9-point
    operator with a unit diagonal: two matvecs of 8 multiplications and 8
    additions (Sec. IV-A: the diagonal's multiply-add earns no credit once
    the diagonal is preconditioned to one), four inner products and six
    AXPYs as in Table I.  The 9-point matvec itself performs 9 fused
    multiply-adds, 18 operations, per point (Sec. IV-A)."""
    matvec = 2 * 8
    return 2 * matvec + 2 * 4 + 2 * 6


def matvec_ops_9pt(with_diagonal=True):
    """Operations of one 9-point matvec per point: 9 multiply-adds (18), or
    16 without the diagonal's."""
    return 18 if with_diagonal else 16


def bytes_per_cell_9pt(w_coef, w_vec, w_x):
    """The fused schedule on the 9-point operator: 8 coefficient words per
    stencil sweep, 16 w_c + 15 w_v + 2 w_x."""
    return 16 * w_coef + 15 * w_vec + 2 * w_x
