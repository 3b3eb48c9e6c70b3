"""The allocation-free filter entry point (vx_filter_device_static) against
the allocating one (vx_filter) and the oracle's filter, through the C ABI, on
two calls in a row.

The entry point serves callers that cannot let a library allocate device
memory (a host framework's memory manager owns all of it, or a cudaMalloc
would stall a latency-critical path): its scratch is a fixed device array
shared by all calls.  The second call runs after the first has left its
counts and offsets in that array, so a stale value used by mistake would
show up as a mismatch.  This file is collected last so that a run stopping at
the first failure has run every other test before it.
"""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")
torch = pytest.importorskip("torch")


def _reference(cols, preds, n):
    """Row ids from the allocating entry point over the same host columns."""
    ctx = vx.vx_open(64 << 20)
    try:
        cfg = vx.vx_get_config(ctx)
        cfg.chunk_bytes = 4 << 20
        vx.vx_set_config(ctx, cfg)
        ids = [vx.vx_register_host_column(ctx, f"c{i}", c) for i, c in enumerate(cols)]
        out = np.zeros(n, np.uint64)
        st, cnt = vx.vx_filter(ctx, [(ids[c], op, lo, hi) for c, op, lo, hi in preds], 0, 0, out)
        assert st == vx.VX_OK
        return out[:cnt]
    finally:
        vx.vx_close(ctx)


def test_static_filter_matches_allocating_filter_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    n = 3_000_001  # ragged: not a multiple of the 2,048-row tile
    f = G.star_fact(n, seed=21)
    cols = [f["quantity"], f["discount"], f["price"]]
    dev = [torch.from_numpy(c).cuda() for c in cols]
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    calls = [
        [(0, vx.VX_LT, 25, 0), (1, vx.VX_BETWEEN, 1, 3)],      # ~13% of rows
        [(2, vx.VX_GE, 9_900_000, 0), (0, vx.VX_NE, 7, 0)],    # ~1% of rows
    ]
    for preds in calls:
        exp = _reference(cols, preds, n)
        # the allocating entry point agrees with the oracle's definition (Section 6.3 selection)
        want = O.filter_rows([(cols[c], op, lo, hi) for c, op, lo, hi in preds], n)
        assert np.array_equal(exp, want)
        out.fill_(-1)
        torch.cuda.synchronize()
        st, cnt = vx.vx_filter_device_static([t.data_ptr() for t in dev], preds, n, 0, out.data_ptr(), n)
        assert st == vx.VX_OK and cnt == len(exp)
        got = out[:cnt].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, exp)
        # nothing written past the count
        assert bool((out[cnt:cnt + 1000] == -1).all())


def test_static_filter_limits():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    col = torch.zeros(10, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(vx.VxError) as e:
        vx.vx_filter_device_static([col.data_ptr()], [(0, vx.VX_EQ, 0, 0)], (1 << 26) + 1, 0, out.data_ptr(), 4)
    assert e.value.status == vx.VX_E_INVAL
    st, cnt = vx.vx_filter_device_static([col.data_ptr()], [(0, vx.VX_EQ, 0, 0)], 10, 100, out.data_ptr(), 4)
    assert st == vx.VX_E_CAPACITY and cnt == 10
    assert out.cpu().tolist() == [100, 101, 102, 103]
