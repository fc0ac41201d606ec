"""The allocation-free compaction entry point, df_active_compact_static.

It serves callers that cannot allocate device memory (a solver whose pool allocator owns the
device, or a path that must not take cudaMalloc's implicit device synchronisation): its
scratch is a static array in the library's device image instead of memory from a df_state.
Its result must be identical to the stateful df_active_compact's, call after call, because
the static scratch is shared and keeps whatever the previous call left in it. This file is
collected last so that a failure here does not hide the rest of the suite."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_compaction_matches_stateful_compaction_twice():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as df
    from paper_2508_18969_gb300 import api
    mech, net, _, _, _ = synth.configs.build("small-fp32-4k", n_cells=8)
    st = df.State(mech, net, T_react=600.0, batch_cells=256)
    # two calls in a row, the second smaller, so entries the first call left in the shared
    # scratch would show up if the second read any it did not write
    for N, seed in ((100003, 1), (77777, 2)):
        T = synth.Stream(seed, "static-compact").uniform(N, 100.0, 1200.0)
        T[3] = np.nan
        Td = torch.tensor(T, device="cuda:0")
        idx_ref, cnt_ref = st.active_compact(Td)
        idx, cnt = api.active_compact_static(Td, 600.0)
        torch.cuda.synchronize()
        c = int(cnt.cpu()[0])
        assert c == int(cnt_ref.cpu()[0]) == int(np.count_nonzero(T > 600.0))
        assert np.array_equal(idx.cpu().numpy()[:c], idx_ref.cpu().numpy()[:c])
