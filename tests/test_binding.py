"""Argument marshalling of the Python binding (CPU): every accepted layout of a block of columns
maps to the pointer, leading dimension and column count the C ABI expects, in the data dtype,
and every other layout or dtype is refused before the library could read outside the buffer."""
import ctypes

import numpy as np
import pytest
import torch


def _read(ptr, ld, ncols, m, dtype):
    """The m x ncols matrix the library would read (column q at ptr + q * ld elements)."""
    n = (ncols - 1) * ld + m
    flat = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype))), (n,))
    return np.stack([flat[q * ld:q * ld + m] for q in range(ncols)], axis=1)


@pytest.mark.parametrize("esize,npd,td", [(4, np.float32, torch.float32), (8, np.float64, torch.float64)])
def test_tensor_layouts(esize, npd, td):
    from paper_2405_16076_gb300.rid import _columns
    m, b = 7, 3
    A = np.arange(m * b, dtype=npd).reshape(m, b) + 0.5            # the m x b block
    cases = [
        torch.from_numpy(np.ascontiguousarray(A.T)).to(td),        # (b, m): row q = column q
        torch.from_numpy(np.ascontiguousarray(A.T)).to(td).T,      # (m, b) column-major view
    ]
    wide = torch.zeros((b, m + 5), dtype=td)
    wide[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T))
    cases.append(wide[:, :m])                                      # rows of a wider matrix: ld = m + 5
    for X in cases:
        ptr, on_dev, ld, ncols, owner = _columns(X, m, esize)
        assert not on_dev and ncols == b and ld >= m
        assert np.array_equal(_read(ptr.value, ld, ncols, m, npd), A)
    one = torch.from_numpy(A[:, 0].copy()).to(td)
    ptr, _, ld, ncols, _ = _columns(one, m, esize)
    assert (ld, ncols) == (m, 1) and np.array_equal(_read(ptr.value, ld, 1, m, npd)[:, 0], A[:, 0])


def test_tensor_refusals():
    from paper_2405_16076_gb300.rid import _columns
    m, b = 7, 3
    with pytest.raises(TypeError):
        _columns(torch.zeros((b, m), dtype=torch.float64), m, 4)
    with pytest.raises(TypeError):
        _columns(torch.zeros((b, m), dtype=torch.float32), m, 8)
    with pytest.raises(ValueError):
        _columns(torch.zeros((b, 2 * m))[:, ::2], m, 4)               # strided coordinates
    with pytest.raises(ValueError):
        _columns(torch.zeros((b, m + 1)), m, 4)                       # no m-long dimension
    with pytest.raises(ValueError):
        _columns(torch.zeros((2, b, m)), m, 4)


@pytest.mark.parametrize("esize,npd", [(4, np.float32), (8, np.float64)])
def test_numpy_layouts_and_conversion(esize, npd):
    from paper_2405_16076_gb300.rid import _columns
    m, b = 7, 3
    A = np.arange(m * b, dtype=np.float64).reshape(m, b) / 8.0     # exact in FP32 too
    cases = [np.asfortranarray(A), np.ascontiguousarray(A.T), np.ascontiguousarray(A),   # the last: copied
             np.asfortranarray(A, dtype=np.float32), A.T.astype(np.float32).tolist()]
    for X in cases:
        ptr, on_dev, ld, ncols, owner = _columns(X, m, esize)
        assert not on_dev and (ld, ncols) == (m, b) and owner.dtype == npd
        assert np.array_equal(_read(ptr.value, ld, ncols, m, npd), A.astype(npd))
    ptr, _, ld, ncols, owner = _columns(A[:, 1], m, esize)
    assert (ld, ncols) == (m, 1) and np.array_equal(_read(ptr.value, ld, 1, m, npd)[:, 0], A[:, 1])
    with pytest.raises(ValueError):
        _columns(np.zeros((b, m + 1)), m, esize)
    with pytest.raises(ValueError):
        _columns(np.zeros((2, b, m)), m, esize)


def test_device_outputs_are_checked_before_any_write():
    from paper_2405_16076_gb300.rid import _device_out
    with pytest.raises(TypeError, match="torch tensor"):
        _device_out(np.zeros(8), "torch.float64", 8, "P")
    with pytest.raises(TypeError, match="float64"):
        _device_out(torch.zeros(8, dtype=torch.float32), "torch.float64", 8, "P")
    with pytest.raises(ValueError, match="contiguous"):
        _device_out(torch.zeros((4, 4), dtype=torch.float64).T, "torch.float64", 8, "P")
    with pytest.raises(ValueError, match="elements"):
        _device_out(torch.zeros(7, dtype=torch.float64), "torch.float64", 8, "P")
    with pytest.raises(TypeError, match="CUDA"):
        _device_out(torch.zeros(8, dtype=torch.float64), "torch.float64", 8, "P")


def test_single_column_views_of_any_stride():
    from paper_2405_16076_gb300.rid import _columns
    m = 9
    v = torch.arange(m, dtype=torch.float32)
    for X in (v, v.unsqueeze(0), v.unsqueeze(1)):
        ptr, _, ld, ncols, _ = _columns(X, m, 4)
        assert ncols == 1 and ld >= m
        assert np.array_equal(_read(ptr.value, ld, 1, m, np.float32)[:, 0], v.numpy())
