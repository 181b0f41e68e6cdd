"""Host-side checks of the Q1 operator descriptor (no GPU): the binding refuses conductivity
arrays of the wrong size or type before any call into the library."""
import numpy as np
import pytest

from paper_2603_09790_gb300 import sstep


def test_q1_descriptor_sizes():
    q = sstep.Q1(5, 4, 3, np.ones((4, 5, 6)))
    assert q.n == 60 and q.ncell == 120


@pytest.mark.parametrize("kappa", [np.ones(119), np.ones(121), np.ones(120, dtype=np.float32)])
def test_q1_rejects_bad_conductivity_arrays(kappa):
    with pytest.raises(ValueError):
        sstep.Solver(sstep.Q1(5, 4, 3, kappa), lambda_max=2.0)
