"""The allocation-free sketch entry point, checked against the plan-based one.

Some callers cannot allocate device memory when they need a sketch -- an
in-situ simulation that has reserved nearly all GPU memory through its own
pool, or one whose time loop must not call cudaMalloc/cudaFree (they may
synchronize the whole device).  spid_sketch_fp32_noalloc serves them: its
split-K partial sums live in a fixed static device array inside the library.
This test calls it through the C ABI twice in a row (the second call on other
data, so stale scratch from the first would show), for every compiled sketch
height (l padded to 16, 32, 48 and 64), and compares each
result with the plan-based FP32 sketch (spid_sketch_accumulate +
spid_get_sketch) and with the FP64 oracle's sketch, within the FP32 sketch
tolerance the parity tests use.  It runs last so that a failure
here cannot hide any other test's result, and it passes both alone in a fresh
process and after the rest of the suite."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_01380_gb300 import inputs, spid

pytestmark = pytest.mark.gpu

Y_TOL_FP32 = 2e-6   # same bound as the FP32 sketch parity tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()


def _plan_sketch(A_dev, m, n, ld, l, seed):
    plan = spid.Plan([m], [n], [0], [ld], k_max=l - 4, p=4, precision="fp32", seed=seed)
    plan.sketch_accumulate(A_dev)
    torch.cuda.synchronize()
    Y = plan.sketches()[0]          # l x n
    plan.close()
    return Y


def _noalloc_sketch(A_dev, m, n, ld, l, seed, ldy):
    Y = torch.full((n * ldy,), float("nan"), dtype=torch.float32, device="cuda")
    spid.sketch_fp32_noalloc(A_dev, m, n, ld, l, seed, Y, ldy)
    torch.cuda.synchronize()
    return Y.cpu().numpy().reshape(n, ldy)[:, :l].T


def _rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("l", [10, 30, 40, 64])
def test_noalloc_sketch_matches_plan_sketch_on_two_calls(l):
    cases = [  # (m, n, seed): ragged rows, two column groups, then a smaller problem
        (5003, 700, 0x5EED0001),
        (1234, 97, 0x5EED0002),
    ]
    for m, n, seed in cases:
        A = inputs.separated_lowrank(m, n, 6, seed=m, noise=1e-3)
        win = inputs.pack_blocks([A])
        A_dev = torch.from_numpy(win.data).cuda()
        ld = int(win.ld[0])
        got = _noalloc_sketch(A_dev, m, n, ld, l, seed, ldy=l + 3)
        assert np.all(np.isfinite(got))
        # the plan-based sketch, where a plan's QR takes the shape (more than
        # 512 columns needs the sketch padded to at most 48 rows)
        if n <= 512 or l <= 48:
            want = _plan_sketch(A_dev, m, n, ld, l, seed)
            assert _rel(got, want) <= Y_TOL_FP32, (m, n, l, _rel(got, want))
        # and the oracle's sketch of the same FP32 values
        Yo = oracle.sketch(win.block(0).astype(np.float64), l, seed)
        assert _rel(got, Yo) <= Y_TOL_FP32, (m, n, l, _rel(got, Yo))


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    lib = spid.load_library()
    A = torch.zeros(64 * 4, dtype=torch.float32, device="cuda")
    Y = torch.zeros(64 * 4, dtype=torch.float32, device="cuda")
    # 129 column groups of 512 columns at l_pad = 32 need 129 * 512 * 32 > 2^21 floats
    n = 129 * 512
    rc = lib.spid_sketch_fp32_noalloc(A.data_ptr(), 4, n, 4, 30, 1, Y.data_ptr(), 30, None)
    assert rc == 1   # SPID_ERR_INVALID_ARG, nothing launched
    assert b"static scratch" in lib.spid_last_error()
