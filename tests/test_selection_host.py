"""Host logic of the model-selection helpers (no GPU): edge counting and the F1 of a
recovered support, checked by hand."""
import types

import numpy as np
import pytest

from paper_1509_04681_gb300 import selection


def test_support_f1_by_hand():
    true = np.array([[2.0, 0.5, 0.0], [0.5, 2.0, 0.3], [0.0, 0.3, 2.0]])
    est = np.array([[1.9, 0.4, 0.1], [0.4, 2.1, 0.0], [0.1, 0.0, 2.0]])
    # Lambda edges (i < j): true {(0,1), (1,2)}, found {(0,1), (0,2)}: tp 1
    s = selection.support_f1(est, true, upper=True)
    assert (s.true_edges, s.found_edges) == (2, 2)
    assert s.precision == 0.5 and s.recall == 0.5 and s.f1 == 0.5
    # with a threshold that drops the 0.1 entry: found {(0,1)}, precision 1, recall 1/2
    s = selection.support_f1(est, true, threshold=0.2, upper=True)
    assert s.precision == 1.0 and s.recall == 0.5 and abs(s.f1 - 2 / 3) < 1e-15
    # all entries (Theta-like): 7 true nonzeros, 7 found, 5 in common
    s = selection.support_f1(est, true)
    assert (s.true_edges, s.found_edges) == (7, 7) and abs(s.f1 - 5 / 7) < 1e-15
    # nothing to find and nothing found
    z = selection.support_f1(np.zeros((2, 2)), np.zeros((2, 2)))
    assert z.precision == 1.0 and z.recall == 1.0 and z.f1 == 1.0
    with pytest.raises(ValueError):
        selection.support_f1(np.zeros((2, 2)), np.zeros((3, 3)))


def test_edge_counts_from_coordinate_lists():
    res = types.SimpleNamespace(
        Lambda_coo=(np.array([0, 0, 1, 1, 2], np.int32), np.array([0, 1, 1, 2, 2], np.int32),
                    np.array([2.0, 0.4, 2.0, -0.3, 2.0])),
        Theta_coo=(np.array([0, 3], np.int32), np.array([1, 0], np.int32), np.array([0.7, -1.0])))
    assert selection.edge_counts(res) == (2, 2)
