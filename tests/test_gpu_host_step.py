"""df_chem_step_host (reaction step of cells in host memory, pipelined through the device in
chunks, or with the kernels reading and writing the host arrays in place) against
df_chem_step on the same cells: every per-cell result is computed by the same kernels with the
same arithmetic, so T, Y and the status bits must agree bit for bit, whatever the chunking;
the step summary covers all chunks."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("chunk,pinned", [(0, True), (7777, True), (0, False), (-1, True)])
def test_host_step_equals_device_step(df, chunk, pinned):
    mech, net, T, p, Y = synth.configs.build("react30-16m", n_cells=300_001)
    st = df.State(mech, net, precision=df.DF_BF16, T_react=600.0, batch_cells=131072)
    dev = torch.device("cuda", 0)
    Td, pd, Yd = (torch.tensor(a, device=dev) for a in (T, p, Y))
    sd = torch.empty(T.shape[0], dtype=torch.int32, device=dev)
    st.chem_step(Td, pd, Yd, status=sd)
    rc_d, n_act_d, n_fl_d, it_d = st.step_summary()
    mk = (lambda a: torch.tensor(a).pin_memory()) if pinned else (lambda a: torch.tensor(a))
    Th, ph, Yh = mk(T), mk(p), mk(Y)
    sh = torch.empty(T.shape[0], dtype=torch.int32)
    if pinned:
        sh = sh.pin_memory()
    st.chem_step_host(Th, ph, Yh, status=sh, chunk_cells=chunk)
    torch.cuda.current_stream().synchronize()
    rc_h, n_act_h, n_fl_h, it_h = st.step_summary()
    assert torch.equal(Th, Td.cpu()) and torch.equal(Yh, Yd.cpu())
    assert torch.equal(sh, sd.cpu())
    assert (n_act_h, n_fl_h, it_h) == (n_act_d, n_fl_d, it_d)
    assert 0 < n_act_h < T.shape[0]
    st.close()


def test_direct_host_access_needs_page_locked_arrays(df):
    """DF_HOST_DIRECT refuses arrays outside page-locked, mapped host memory before any device
    work, and leaves them untouched."""
    mech, net, T, p, Y = synth.configs.build("react30-16m", n_cells=5000)
    st = df.State(mech, net, precision=df.DF_BF16, T_react=600.0, batch_cells=4096)
    Th, Yh = torch.tensor(T).pin_memory(), torch.tensor(Y).pin_memory()
    ph = torch.tensor(p)   # pageable
    with pytest.raises(df.DFError, match="DF_HOST_DIRECT"):
        st.chem_step_host(Th, ph, Yh, chunk_cells=df.DF_HOST_DIRECT)
    sh = torch.empty(T.shape[0], dtype=torch.int32)   # pageable status
    with pytest.raises(df.DFError, match="DF_HOST_DIRECT"):
        st.chem_step_host(Th, ph.pin_memory(), Yh, status=sh, chunk_cells=df.DF_HOST_DIRECT)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(Th, torch.tensor(T)) and torch.equal(Yh, torch.tensor(Y))
    st.close()
