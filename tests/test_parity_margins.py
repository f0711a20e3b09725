"""The float64 parity cases compare the GPU's augmented ranks with the oracle's bit for
bit.  That comparison is well posed only when no fill singular value sits within
rounding of the threshold eps_fill = eps_lu ||A|| (Alg. 2 keeps sigma > eps_fill), where
two correct float64 computations could round to different ranks.  This checks, with
the oracle alone, that every truncation decision of every float64 parity case has a
relative margin of at least 1e-8."""
import numpy as np
import pytest

from oracle import rs

from conftest import problem
from test_gpu_parity import CASES, IDS

MARGIN = 1e-8


@pytest.mark.parametrize("name,over,eps", CASES, ids=IDS)
def test_no_fill_singular_value_at_the_threshold(name, over, eps):
    pb = problem(name, **over)
    A = pb.A.numpy()
    eps_fill = eps * pb.norm_a
    gaps = []

    def hook(stage, **kw):
        if stage != "augment" or kw["Frow"] is None:
            return
        V, Frow = kw["V"], kw["Frow"]
        if V.shape[1] >= V.shape[0] or Frow.shape[1] == 0:
            return
        Y = Frow - V @ (V.T @ Frow)
        s = np.linalg.svd(Y, compute_uv=False)
        gaps.append(np.min(np.abs(s / eps_fill - 1.0)))

    rs.factorize(A, eps, pb.norm_a, hook=hook)
    assert gaps, "no truncation decision was made"
    assert min(gaps) > MARGIN, min(gaps)
