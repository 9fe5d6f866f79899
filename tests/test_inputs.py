"""The seeded input generators: Gaussian moments (Sec. 3) and Haar structure."""
import numpy as np

from paper_2008_04447_gb300 import inputs as I


def test_omega_sketch_moments():
    """E||Omega a||^2 = l ||a||^2 and Var = 2 l ||a||^4 for GIID Omega (Sec. 3)."""
    l, m, trials = 12, 30, 20000
    g = I.rng(5)
    a = g.standard_normal(m)
    a2 = a @ a
    vals = np.empty(trials)
    for t in range(0, trials, 1000):
        om = I.omega(l, m, seed=10_000 + t).reshape(l, m)
        # 1000 independent draws per seed by re-slicing fresh Gaussians
        w = I.rng(20_000 + t).standard_normal((1000, l, m))
        vals[t:t + 1000] = np.sum((w @ a) ** 2, axis=1)
    mean = vals.mean()
    var = vals.var()
    assert abs(mean / (l * a2) - 1) < 0.03
    assert abs(var / (2 * l * a2 ** 2) - 1) < 0.08


def test_haar_and_graded():
    q = I.haar(50, 20, I.rng(1))
    assert np.allclose(q.T @ q, np.eye(20), atol=1e-13)
    a = I.graded(40, 30, 8, seed=2)
    s = np.linalg.svd(a, compute_uv=False)
    assert np.allclose(s, 10.0 ** (-8 * np.arange(1, 31) / 30), rtol=1e-6)
    assert np.array_equal(I.graded(40, 30, 8, seed=2), a)


def test_batch_shapes():
    sh = I.batch_shapes(500, seed=0)
    for m, n, k in sh:
        assert 64 <= m <= 2048 and 1 <= n <= min(m, 1024) and 1 <= k <= min(m, n) // 2


def test_lowrank_parts_rebuild_the_matrix_exactly():
    """The parts (Haar U, sigma_i = i^-2, Haar V, noise) come from the same
    generator in the same order as the matrix itself, so (U s) V^T + noise
    reproduces it bit for bit (the full-size TUXV test relies on it)."""
    import torch
    from paper_2008_04447_gb300 import inputs as I
    for args in [(300, 200, 64, 1e-6, 7), (120, 90, 200, 0.0, 3)]:
        a = I.lowrank_plus_noise_torch(*args, device="cpu")
        u, s, v, nz = I.lowrank_plus_noise_parts_torch(*args, device="cpu")
        b = (u * s) @ v.T
        if nz is not None:
            b += nz
        assert torch.equal(a, b)
        assert (nz is None) == (args[3] == 0.0)
        assert torch.equal(s, torch.arange(1, s.numel() + 1, dtype=torch.float64) ** -2.0)
