"""The repository's smoke check (one small apply in each precision and one mixed BVP solve
on cuda:0, each against the oracle) run as a GPU test, so that the suite covers it too."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import __graft_entry__ as G
    G.smoke()
