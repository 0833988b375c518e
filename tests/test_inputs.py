"""The device-side field generator reproduces the host generator (CPU torch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_01380_gb300 import inputs


def test_device_field_matches_host_boxes():
    modes = inputs.fourier_modes(seed=2)
    origins = [(0, 0, 0), (24, 8, 28)]          # the second box wraps around the grid
    t = 10.0 * np.arange(12) / 11.0
    f = inputs.DeviceField(origins, 8, 32, modes, device="cpu")
    got = f.snapshots(t).numpy()                 # [5, S*P, n]
    for s, o in enumerate(origins):
        want = inputs.tgv3d_box(o, (8, 8, 8), 32, t, modes, dtype=np.float64)
        P = 512
        blk = got[:, s * P:(s + 1) * P, :].reshape(5 * P, len(t))
        np.testing.assert_allclose(blk, want, rtol=2e-5, atol=2e-5 * np.abs(want).max())


def test_snapshot_major_fill_layout():
    modes = inputs.fourier_modes(seed=2)
    origins = [(0, 0, 0), (8, 0, 0), (0, 8, 0)]
    n = 6
    t = 10.0 * np.arange(n) / (n - 1)
    f = inputs.DeviceField(origins, 8, 16, modes, device="cpu")
    m = 5 * 512
    window = torch.zeros(n * 3 * m, dtype=torch.float32)
    f.fill_snapshot_major(window, t[:4], 0, n)
    f.fill_snapshot_major(window, t[4:], 4, n)
    w = inputs.Window(window.numpy(), np.full(3, m), np.full(3, n), np.arange(3) * m,
                      np.full(3, 3 * m))
    for s, o in enumerate(origins):
        want = inputs.tgv3d_box(o, (8, 8, 8), 16, t, modes, dtype=np.float64)
        np.testing.assert_allclose(w.block(s), want, rtol=2e-5, atol=2e-5 * np.abs(want).max())
