"""The Python binding's element-count checks, which stand between a wrong-sized array and the C
ABI's plain pointers.  A Context is built without a device (its pointer is never used: every case
fails before the library is called), so this runs on CPU."""
import numpy as np
import pytest

from paper_2505_22718_gb300.api import Context, _need


def _ctx():
    c = Context.__new__(Context)
    c.ptr = None
    c.N, c.n_k, c.n_ell, c.n_knots, c.n_tr = 64, 10, 5, 3, 2
    c.n_walk, c.n_out = 1, 5
    return c


def test_need_counts_numpy_lists_and_tensors():
    torch = pytest.importorskip("torch")
    _need(np.zeros((2, 3)), 6, "x")
    _need([1.0, 2.0], 2, "x")
    _need(torch.zeros(4, 2), 8, "x")
    _need(None, 3, "x")
    _need(np.zeros(5), None, "x")
    with pytest.raises(ValueError, match="has 5 elements, expected 6"):
        _need(np.zeros(5), 6, "x")


def test_context_rejects_wrong_sizes_before_calling_the_library():
    c = _ctx()
    with pytest.raises(ValueError, match="W"):
        c.set_windows(np.zeros((2, 63)))
    with pytest.raises(ValueError, match="D"):
        c.set_windows(np.zeros((2, 64)), np.zeros((2, 64)))
    with pytest.raises(ValueError, match="B"):
        c.set_windows(np.zeros((2, 64)), np.zeros((3, 64)), np.zeros((2, 3, 32)))
    with pytest.raises(ValueError, match="W"):
        c.set_windows(np.zeros((4, 2, 32)))        # four walkers of the wrong length
    with pytest.raises(ValueError, match="P"):
        c.set_power(np.zeros(9), np.zeros(2))
    with pytest.raises(ValueError, match="amp"):
        c.set_power(np.zeros(10), np.zeros(3))
    with pytest.raises(ValueError, match="C_out"):
        c.compute_cl(out=np.zeros((4, 2, 2)))
    with pytest.raises(ValueError, match="C_bar"):
        c.vjp(np.zeros((5, 2, 3)))
    with pytest.raises(ValueError, match="P_dot"):
        c.jvp(P_dot=np.zeros((2, 11)))
    with pytest.raises(ValueError, match="W_dot"):
        c.jvp(W_dot=np.zeros((1, 2, 32)))
    with pytest.raises(ValueError, match="modes"):
        c.gaussian_fisher(np.zeros((1, 5, 2, 2)), np.zeros(4))
    with pytest.raises(ValueError, match="noise"):
        c.gaussian_fisher(np.zeros((1, 5, 2, 2)), np.zeros(5), np.zeros(3))


def test_unset_shapes_are_not_checked():
    c = _ctx()
    c.n_knots = 0                      # before set_grids: left to the library's own state check
    assert c._shape(c.n_knots, c.N) is None
    assert c._shape(2, 3, 4) == 24
