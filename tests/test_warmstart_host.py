"""Host-side logic of the learned warm start (CPU): the feature scaling the
network's inputs are normalised with."""
import numpy as np

from paper_1802_08557_gb300 import workloads as W
from paper_1802_08557_gb300.warmstart import feature_scaling


def test_feature_scaling_is_mean_and_inverse_std_of_b_and_c():
    B = W.shared_matrix_family(500, m=20, n=10)
    mean, inv = feature_scaling(B)
    f = np.concatenate([B.b.reshape(500, 20), B.c.reshape(500, 10)], axis=1)
    assert mean.dtype == np.float32 and inv.dtype == np.float32 and mean.shape == (30,)
    np.testing.assert_allclose(mean, f.mean(axis=0), rtol=1e-6)
    np.testing.assert_allclose(inv, 1.0 / f.std(axis=0), rtol=1e-6)
    # scaled features: mean 0, std 1 per feature
    z = (f - mean) * inv
    np.testing.assert_allclose(z.mean(axis=0), 0.0, atol=1e-4)
    np.testing.assert_allclose(z.std(axis=0), 1.0, rtol=1e-4)


def test_feature_scaling_constant_feature_gets_unit_scale():
    B = W.shared_matrix_family(50, m=6, n=4)
    c = B.c.reshape(50, 4)
    c[:, 2] = 0.25  # a cost that never changes
    mean, inv = feature_scaling(B)
    assert mean[6 + 2] == np.float32(0.25) and inv[6 + 2] == 1.0
    assert np.all(np.isfinite(inv))


def test_feature_scaling_samples_large_batches_evenly():
    """Above 20000 LPs the statistics come from every (N // 20000)-th LP."""
    B = W.shared_matrix_family(40_000, m=3, n=2)
    mean, inv = feature_scaling(B)
    f = np.concatenate([B.b.reshape(-1, 3), B.c.reshape(-1, 2)], axis=1)[::2]
    np.testing.assert_allclose(mean, f.mean(axis=0), rtol=1e-6)
    np.testing.assert_allclose(inv, 1.0 / f.std(axis=0), rtol=1e-5)
