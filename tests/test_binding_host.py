"""CPU: the binding's layout helpers on degenerate shapes.

``colmajor`` must give stride 1 between rows of every 2-D tensor, and ``_ld``
must return the leading dimension the C ABI expects (entry (i, j) at
i + j ld, ld >= max(1, rows)), including single-row and single-column
matrices, whose size-1 dimension carries an arbitrary stride in torch.
"""
import pytest
import torch

from paper_2008_04447_gb300 import _ld, colmajor


@pytest.mark.parametrize("shape", [(1, 5), (5, 1), (1, 1), (3, 4), (7, 2)])
def test_colmajor_places_entry_ij_at_i_plus_j_ld(shape):
    x = torch.arange(shape[0] * shape[1], dtype=torch.float64).reshape(shape)
    c = colmajor(x)
    assert torch.equal(c, x)
    ld = _ld(c)
    assert ld >= max(1, shape[0])
    flat = torch.as_strided(c, (ld * (shape[1] - 1) + shape[0],), (1,))
    for i in range(shape[0]):
        for j in range(shape[1]):
            assert float(flat[i + j * ld]) == float(x[i, j])


def test_single_row_with_row_major_strides_is_accepted():
    x = torch.randn(1, 6)                       # strides (6, 1)
    assert x.stride() == (6, 1)
    assert _ld(x) == 1                          # entry (0, j) at j * 1
    y = torch.randn(8, 6)[2:3, :]               # a row of a row-major matrix: strides (6, 1)
    assert _ld(y) == 1
    z = torch.randn(6, 8).t()[3:4, :]           # a row of a column-major 8 x 6 matrix: column stride 8
    assert _ld(z) == 8


def test_row_major_matrix_is_rejected():
    with pytest.raises(ValueError):
        _ld(torch.randn(3, 4))
    with pytest.raises(ValueError):
        _ld(torch.randn(4))


def test_single_column_keeps_ld_at_least_rows():
    x = torch.randn(5, 1)                       # strides (1, 1)
    assert _ld(x) == 5
    assert _ld(colmajor(x)) == 5
