"""The binding rejects vectors of the wrong length before any pointer reaches
the C ABI (the kernels and host copies read exactly n entries, so a short
vector would be read past its end).  No GPU and no library call needed: the
checks run first, and load_library is replaced by a tripwire."""
import types

import numpy as np
import pytest

import paper_1609_09068_gb300 as prgb


@pytest.fixture
def no_library(monkeypatch):
    def tripwire():
        raise AssertionError("the C library was reached")
    monkeypatch.setattr(prgb, "load_library", tripwire)


def _part(n, n_comp):
    return types.SimpleNamespace(n=n, n_comp=n_comp, handle=None)


def test_solve_rejects_short_u(no_library):
    with pytest.raises(ValueError, match="u has 9 entries, expected 10"):
        prgb.solve(_part(10, 3), 0.85, np.ones(9), 1e-10)


def test_solve_rejects_long_u_on_host(no_library):
    with pytest.raises(ValueError, match="u has 11 entries"):
        prgb.solve(_part(10, 3), 0.85, np.ones(11), 1e-10)


def test_solve_rejects_short_replay(no_library):
    with pytest.raises(ValueError, match="replay_iters has 2 entries, expected 3"):
        prgb.solve(_part(10, 3), 0.85, np.ones(10), 1e-10, replay_iters=[5, 5])


def test_solve_rejects_matrix_u(no_library):
    with pytest.raises(ValueError, match="1-D"):
        prgb.solve(_part(10, 3), 0.85, np.ones((10, 1)), 1e-10)


def test_global_and_residual_reject_short_vectors(no_library):
    g = types.SimpleNamespace(n=10, handle=None)
    with pytest.raises(ValueError, match="u has 4 entries"):
        prgb.global_power(g, 0.85, np.ones(4), 1e-10)
    with pytest.raises(ValueError, match="R has 8 entries"):
        prgb.residual_l1(g, 0.85, np.ones(10), np.ones(8))


def test_static_residual_rejects_short_vectors(no_library):
    rowptr = np.zeros(11, np.int32)
    col = np.zeros(0, np.int32)
    with pytest.raises(ValueError, match="u has 3 entries, expected 10"):
        prgb.residual_l1_static(rowptr, col, 0.85, np.ones(3), np.ones(10))
    with pytest.raises(ValueError, match="R has 12 entries"):
        prgb.residual_l1_static(rowptr, col, 0.85, np.ones(10), np.ones(12))


def test_mpnn_calls_reject_short_vectors(no_library):
    m = object.__new__(prgb.Mpnn)  # no device model: the check comes first
    p = _part(10, 3)
    for fn in (m.predict, m.loss_grad, m.train_step):
        with pytest.raises(ValueError, match="u has 9 entries"):
            fn(p, 0.85, np.ones(9), np.ones(10))
        with pytest.raises(ValueError, match="R has 7 entries"):
            fn(p, 0.85, np.ones(10), np.ones(7))


def test_load_partition_takes_a_graph(no_library, tmp_path):
    with pytest.raises(TypeError, match="takes a Graph"):
        prgb.load_partition(np.zeros(3, np.int32), tmp_path / "p.bin")
