"""The in-situ producer (spid_producer_step, a stand-in for the paper's flow
solver used to measure compression next to a running solver) against a numpy
restatement of its update on the global periodic grid: first-order upwind
advection by the velocity QoIs 1..3 plus nu times the 7-point Laplacian,
forward Euler.  FP32 on the GPU vs FP64 here: a few ulps of the state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_01380_gb300 import spid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()


def to_global(state, grid, edge, nq):
    nb = grid // edge
    s = state.reshape(nb, nb, nb, nq, edge, edge, edge)          # [bz, by, bx, q, z, y, x]
    return s.transpose(3, 0, 4, 1, 5, 2, 6).reshape(nq, grid, grid, grid)   # [q, Z, Y, X]


def to_boxes(field, grid, edge, nq):
    nb = grid // edge
    f = field.reshape(nq, nb, edge, nb, edge, nb, edge)          # [q, bz, z, by, y, bx, x]
    return f.transpose(1, 3, 5, 0, 2, 4, 6).reshape(-1)


def reference_step(F, dt, nu):
    nq, G = F.shape[0], F.shape[1]
    h = 2.0 * np.pi / G
    vel = [F[1], F[2], F[3]]
    out = np.empty_like(F)
    for q in range(nq):
        f = F[q]
        adv = np.zeros_like(f)
        lap = -6.0 * f
        for ax, u in zip((2, 1, 0), vel):                # X, Y, Z axes of [Z, Y, X]
            fm = np.roll(f, 1, axis=ax)
            fp = np.roll(f, -1, axis=ax)
            adv += np.where(u > 0, u * (f - fm), u * (fp - f))
            lap += fm + fp
        out[q] = f - dt / h * adv + nu * dt / h ** 2 * lap
    return out


def test_producer_step_between_window_layouts():
    # the same step read from a snapshot-major state and written into column j
    # of a subdomain-major window ([box][j][rows], box stride nq edge^3 n)
    grid, edge, nq, n, j = 16, 8, 5, 3, 1
    rng = np.random.default_rng(7)
    F = rng.uniform(-1.0, 1.0, size=(nq, grid, grid, grid))
    be = nq * edge ** 3
    nbox = (grid // edge) ** 3
    state = torch.tensor(to_boxes(F, grid, edge, nq), dtype=torch.float32, device="cuda")
    win = torch.zeros(nbox * n * be, dtype=torch.float32, device="cuda")
    spid.producer_step(state, win[j * be:], grid, edge, nq, 0.002, 0.01,
                       out_box_stride=n * be)
    ref = torch.empty_like(state)
    spid.producer_step(state, ref, grid, edge, nq, 0.002, 0.01)
    torch.cuda.synchronize()
    got = win.view(nbox, n, be)[:, j, :].reshape(-1)
    assert torch.equal(got, ref)
    assert float(win.view(nbox, n, be)[:, 0, :].abs().max()) == 0.0   # other columns untouched


@pytest.mark.parametrize("grid,edge,nq", [(16, 8, 5), (12, 4, 4), (8, 8, 5)])
def test_producer_step_matches_the_stencil(grid, edge, nq):
    rng = np.random.default_rng(grid + edge)
    F = rng.uniform(-1.0, 1.0, size=(nq, grid, grid, grid))
    dt, nu = 0.002, 0.01
    state = torch.tensor(to_boxes(F, grid, edge, nq), dtype=torch.float32, device="cuda")
    out = torch.empty_like(state)
    spid.producer_step(state, out, grid, edge, nq, dt, nu)
    # two more steps through a ping-pong pair
    out2 = torch.empty_like(state)
    spid.producer_step(out, out2, grid, edge, nq, dt, nu)
    torch.cuda.synchronize()
    F32 = to_global(state.cpu().numpy().astype(np.float64), grid, edge, nq)
    want1 = reference_step(F32, dt, nu)
    got1 = to_global(out.cpu().numpy().astype(np.float64), grid, edge, nq)
    assert np.max(np.abs(got1 - want1)) <= 1e-5 * np.abs(want1).max()
    want2 = reference_step(got1, dt, nu)
    got2 = to_global(out2.cpu().numpy().astype(np.float64), grid, edge, nq)
    assert np.max(np.abs(got2 - want2)) <= 1e-5 * np.abs(want2).max()
