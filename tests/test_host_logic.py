"""Host-side logic of the drivers that needs no GPU: the training-window sampler of the learned
closure driver and the spectral summaries of the LES-vs-DNS driver."""
import numpy as np
import torch

from paper_1705_09807_gb300.learned_closure import random_crops
from paper_1705_09807_gb300.les_dns import fitted_slope, spectral_errors


def test_random_crops_take_the_same_window_of_features_and_targets():
    X = torch.arange(3 * 12 * 20 * 24, dtype=torch.float32).reshape(3, 12, 20, 24)
    T = -torch.arange(3 * 4 * 20 * 24, dtype=torch.float32).reshape(3, 4, 20, 24)
    xb, tb = random_crops(X, T, 5, 8, np.random.default_rng(3))
    assert xb.shape == (5, 12, 8, 8) and tb.shape == (5, 4, 8, 8)
    assert xb.is_contiguous() and tb.is_contiguous()
    for b in range(5):
        # locate the crop in X from its first element, then check both tensors element-wise
        v = int(xb[b, 0, 0, 0])
        i, rem = divmod(v, 12 * 20 * 24)
        y0, x0 = divmod(rem, 24)
        assert 0 <= y0 <= 12 and 0 <= x0 <= 16
        assert torch.equal(xb[b], X[i, :, y0:y0 + 8, x0:x0 + 8])
        assert torch.equal(tb[b], T[i, :, y0:y0 + 8, x0:x0 + 8])


def test_fitted_slope_and_spectral_errors():
    k = np.arange(64, dtype=np.float64)
    e = np.zeros(64)
    e[1:] = 3.0 * k[1:] ** -2.5
    assert abs(fitted_slope(e, 2, 30) + 2.5) < 1e-12
    rel, logrms = spectral_errors(2.0 * e, e, 40)
    assert abs(rel - 1.0) < 1e-12 and abs(logrms - np.log10(2.0)) < 1e-12
    assert spectral_errors(e, e, 40) == (0.0, 0.0)
