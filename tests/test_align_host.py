"""Host-side pieces of the alignment solver (no GPU): the per-sector 3x3
block inverse used as the conjugate-gradient preconditioner."""
import numpy as np
import torch

from paper_2002_11529_gb300.align import _block_inverse


def test_block_inverse_matches_numpy_and_zeroes_empty_sectors():
    rng = np.random.default_rng(0)
    m = rng.normal(size=(64, 3, 3))
    # scales like the Gauss-Newton blocks: dx ~ 1e2, dz ~ 1e4, gamma ~ 1e8
    h = m @ m.transpose(0, 2, 1) + np.diag([1e2, 1e4, 1e8])
    h6 = np.stack([h[:, 0, 0], h[:, 0, 1], h[:, 0, 2], h[:, 1, 1], h[:, 1, 2], h[:, 2, 2]], 1)
    h6[[5, 17]] = 0.0                                     # sectors without hits
    inv = _block_inverse(torch.from_numpy(h6)).numpy()
    ref = np.linalg.inv(h)
    ref[[5, 17]] = 0.0
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True) + 1e-300
    assert np.max(np.abs(inv - ref) / scale) < 1e-12
    assert np.all(inv[[5, 17]] == 0.0)
    # inverse times block is the identity on the used sectors
    used = np.ones(64, bool)
    used[[5, 17]] = False
    eye = np.einsum("sij,sjk->sik", inv[used], h[used])
    assert np.allclose(eye, np.eye(3)[None], atol=1e-9)
