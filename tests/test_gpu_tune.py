"""Width tuner (gks_tune): picks one of the candidates, applies it to later solves of the
same shape class only, keeps parity with the oracle, and rejects invalid widths."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2606_09058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gks_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks
    return gks


def test_tune_picks_a_candidate_and_solves_match_oracle(gks_mod):
    ctx = gks_mod.Context(0)
    best, ms = ctx.tune(300, nk=2, complex_=True, widths=(64, 128, 192))
    assert best in (64, 128, 192) and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    assert ctx.tune_get(300, True) == best        # same bucket (257..512)
    assert ctx.tune_get(290, True) == best
    assert ctx.tune_get(600, True) == 256         # other bucket: the default
    assert ctx.tune_get(300, False) == 256        # other element type
    H, S = I.random_pencil(311, 77, True, cond=1e2)
    sol = ctx.solve(torch.as_tensor(H[None]).cuda(), torch.as_tensor(S[None]).cuda(), 0.1, 0.6 * 311)
    ref = O.solve(H[None], S[None], 0.1, 0.6 * 311)
    assert np.abs(sol.eps.cpu().numpy() - ref.eps).max() <= 1e-10 * max(1.0, np.abs(ref.eps).max())


def test_tune_set_get_and_invalid(gks_mod):
    ctx = gks_mod.Context(0)
    ctx.tune_set(1000, False, "collinear", 384)
    assert ctx.tune_get(1000, False) == 384
    ctx.tune_set(1000, False, "collinear", 0)
    assert ctx.tune_get(1000, False) == 256
    with pytest.raises(gks_mod.GKSError):
        ctx.tune_set(1000, False, "collinear", 100)
    with pytest.raises(gks_mod.GKSError):
        ctx.tune(200, widths=(96,))
