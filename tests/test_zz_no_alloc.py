"""The allocation-free RV(r) entry point agrees with bc_rv_compute.

Some callers of this library cannot allocate device memory: code running
inside another framework's allocator hooks or teardown, processes whose
device memory is fully reserved by a caching allocator, plugins that are
handed a stream and their buffers but no right to allocate. For them the
library offers bc_rv_compute_noalloc, which works in one fixed file-scope
device array instead of allocating. This test calls it through the C ABI
several times in a row (a large reach set, an empty one, the large one
again, so that leftovers of a previous call would show) and checks every
result against bc_rv_compute, element by element. The test itself allocates
the device inputs and outputs; the call under test allocates nothing.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


def test_noalloc_rv_matches_rv_compute():
    torch = pytest.importorskip("torch")
    import paper_1708_08739_gb300 as bcd

    g = gg.rmat(16, 8, seed=5)
    dg = bcd.bc_graph_create(g.n, g.offsets, g.cols)
    roff, rcol, _ = bcd.bc_graph_reverse(dg)
    d_roff = torch.from_numpy(roff).cuda()
    d_rcol = torch.from_numpy(rcol.copy()).cuda()
    out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    top = int(gg.top_inout_vertices(g, 1)[0])
    empty = int(np.flatnonzero(g.in_degree() == 0)[0])
    small = int(gg.random_vertices(g.n, 1, 9)[0])
    for r in [top, empty, top, small]:
        k = bcd.bc_rv_compute_noalloc(d_roff.data_ptr(), d_rcol.data_ptr(), g.n, r, out.data_ptr(), g.n, stream)
        want = bcd.bc_rv_compute(dg, r)
        got = out[:k].cpu().numpy()
        assert k == want.shape[0], (r, k, want.shape[0])
        assert np.array_equal(got, want), r

    # the stated maximum and the capacity are enforced with clear errors
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_rv_compute_noalloc(d_roff.data_ptr(), d_rcol.data_ptr(), bcd.BC_NOALLOC_MAX_VERTICES + 1, 0,
                                  out.data_ptr(), g.n, stream)
    assert e.value.status == bcd.BC_E_INVALID_ARG
    with pytest.raises(bcd.BCError) as e:
        bcd.bc_rv_compute_noalloc(d_roff.data_ptr(), d_rcol.data_ptr(), g.n, top, out.data_ptr(), 3, stream)
    assert e.value.status == bcd.BC_E_BUFFER_TOO_SMALL
    dg.close()
