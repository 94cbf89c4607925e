"""Host-side rules of the learned pose selector."""
import numpy as np

from paper_2304_09953_gb300 import native as N
from paper_2304_09953_gb300 import selector as S


def test_labels():
    r = np.zeros(4, N.RESCORED_DTYPE)
    r["energy"] = [-3.0, 50.0, -1.0, np.inf]
    r["pass"] = [1, 1, 0, 0]
    np.testing.assert_array_equal(S.labels(r), [-3.0, 30.0, 30.0, 30.0])


def test_select_first_predicted_pass_in_docking_order():
    pred = np.array([[20.0, 3.0, -5.0], [40.0, 35.0, 29.0], [1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    live = np.array([[1, 1, 1], [1, 1, 1], [0, 1, 1], [0, 0, 0]], bool)
    np.testing.assert_array_equal(S.select(pred, live), [1, 2, 1, -1])
