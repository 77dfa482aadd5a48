"""CPU checks of the allocation-free entry point's Python argument checks: a
mismatched shape or a tensor off the current CUDA device is refused with
ValueError before the library is called (so nothing is ever launched with a
short buffer)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11547_gb300 import rot_vote as rv  # noqa: E402


def _args(n=5, nb=None, nc=4, ncount=None, device="cpu"):
    a = torch.zeros((n, 3), dtype=torch.float32, device=device)
    b = torch.zeros((n if nb is None else nb, 3), dtype=torch.float32, device=device)
    cells = torch.zeros(nc, dtype=torch.int64, device=device)
    counts = torch.zeros(nc if ncount is None else ncount, dtype=torch.int32, device=device)
    return a, b, cells, counts


def test_short_b_is_refused():
    with pytest.raises(ValueError, match="a and b"):
        rv.count_cells_static(*_args(nb=4)[:2], 0.03, 8, *_args()[2:])


def test_short_counts_is_refused():
    a, b, cells, _ = _args()
    with pytest.raises(ValueError, match="cells and counts"):
        rv.count_cells_static(a, b, 0.03, 8, cells, _args(ncount=3)[3])


def test_wrong_rank_is_refused():
    a = torch.zeros(15, dtype=torch.float32)
    with pytest.raises(ValueError, match="a and b"):
        rv.check_static_args(a, a, *_args()[2:])


def test_host_tensors_are_refused():
    with pytest.raises(ValueError, match="CUDA device"):
        rv.check_static_args(*_args())
