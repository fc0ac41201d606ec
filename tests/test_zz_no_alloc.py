"""The allocation-free compaction entry point, df_active_compact_static.

It serves callers that cannot allocate device memory (a solver whose pool allocator owns the
device, or a path that must not take cudaMalloc's implicit device synchronisation): its
scratch is a static array in the library's device image instead of memory from a df_state.
Its result must be identical to the stateful df_active_compact's and to the plain list of
reacting cells, call after call, because the static scratch is shared and keeps whatever the
previous call left in it. This file is collected last so that a failure here does not hide
the rest of the suite."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_REACT = 600.0


def _field(N, seed):
    """N temperatures in [100, 1200] K: a seeded block of up to 2^20 values repeated, with a
    NaN, an infinity and a value exactly at the threshold planted in every block."""
    blk = min(N, 1 << 20)
    base = synth.Stream(seed, "static-compact").uniform(blk, 100.0, 1200.0)
    if blk > 10:
        base[3], base[5], base[7] = np.nan, T_REACT, np.inf
    return np.tile(base, (N + blk - 1) // blk)[:N]


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    return m


def test_static_compaction_matches_stateful_compaction_and_the_list(df):
    from paper_2508_18969_gb300 import api
    mech, net, _, _, _ = synth.configs.build("small-fp32-4k", n_cells=8)
    st = df.State(mech, net, T_react=T_REACT, batch_cells=256)
    max_cells = int(df._lib.DF_COMPACT_STATIC_MAX_CELLS)
    # calls in a row, each smaller than the one before, so entries an earlier call left in the
    # shared scratch would show up if a later one read any it did not write. The largest runs
    # the single-block scan over the most chunk counts the array holds; 4 * 2^20 + 4097 cells
    # make a ragged last chunk beyond the scan's one-count-per-thread range.
    for N, seed in ((max_cells, 3), ((4 << 20) + 4097, 4), (100003, 1), (77777, 2)):
        T = _field(N, seed)
        Td = torch.tensor(T, device="cuda:0")
        idx_ref, cnt_ref = st.active_compact(Td)
        idx, cnt = api.active_compact_static(Td, T_REACT)
        torch.cuda.synchronize()
        want = np.flatnonzero(T > T_REACT)
        c = int(cnt.cpu()[0])
        assert c == int(cnt_ref.cpu()[0]) == want.size, N
        got = idx.cpu().numpy()[:c]
        assert np.array_equal(got, want.astype(np.int32)), N
        assert np.array_equal(got, idx_ref.cpu().numpy()[:c]), N
        del Td, idx, idx_ref
    st.close()
    torch.cuda.empty_cache()


def test_static_compaction_rejects_oversize_calls(df):
    """n_cells above the static array's limit is refused on the host, before any launch."""
    lib = df._lib.load()
    T = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    idx = torch.zeros(8, dtype=torch.int32, device="cuda:0")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    rc = lib.df_active_compact_static(int(df._lib.DF_COMPACT_STATIC_MAX_CELLS) + 1, T_REACT,
                                      ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                                      ctypes.c_void_p(cnt.data_ptr()), None)
    assert rc == df._lib.DF_ERR_INVALID_ARG
    assert b"DF_COMPACT_STATIC_MAX_CELLS" in lib.df_get_last_error(None)
