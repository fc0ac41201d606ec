"""Failure handling of the tensor-core kernels without a fault: every pipeline wait of
tc_gemm_kernel is bounded, and df_set_wait_limit shortens the bound so far (a few hundred SM
clocks, less than one TMA load from HBM takes) that the waits run out on purpose. The kernels
must then give up cleanly -- error flag set, copies and MMAs in flight drained, tensor memory
freed -- df_get_step_summary must report DF_ERR_TIMEOUT once, and the state must stay usable.

The layers run on single CTAs here (DFGB_BN forces single-CTA tiles): their way out has no
cluster barrier, so nothing on it can wait for a peer."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    return m


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_short_wait_limit_times_out_and_the_state_recovers(df, prec, monkeypatch):
    monkeypatch.setenv("DFGB_BN", "224")
    mech, net, T, p, Y = synth.configs.build("layer1d-30sp-1m", n_cells=65536)
    P = df.DF_BF16 if prec == "bf16" else df.DF_FP8_E4M3
    st = df.State(mech, net, precision=P, T_react=0.0, batch_cells=65536)
    assert not any(t & df.DF_TILE_PAIR for t in st.tiles()), st.tiles()
    pd = _dev(p)

    st.set_wait_limit(200)
    T0, Y0 = _dev(T), _dev(Y)
    st.chem_step(T0, pd, Y0)
    rc, n_act, _, _ = st.step_summary()
    assert rc == df._lib.DF_ERR_TIMEOUT, rc
    assert n_act == T.shape[0]
    # reported once: the flag is cleared by the summary that reported it
    st.chem_step(T0, pd, Y0)
    rc_again, _, _, _ = st.step_summary()
    assert rc_again == df._lib.DF_ERR_TIMEOUT   # the short limit still applies

    st.set_wait_limit(0)
    T1, Y1 = _dev(T), _dev(Y)
    st.chem_step(T1, pd, Y1)
    rc1, _, f1, _ = st.step_summary()
    fresh = df.State(mech, net, precision=P, T_react=0.0, batch_cells=65536)
    T2, Y2 = _dev(T), _dev(Y)
    fresh.chem_step(T2, pd, Y2)
    rc2, _, f2, _ = fresh.step_summary()
    torch.cuda.synchronize()
    assert rc1 == rc2 != df._lib.DF_ERR_TIMEOUT and f1 == f2
    assert torch.equal(T1, T2) and torch.equal(Y1, Y2)
    assert not torch.equal(Y1, _dev(Y))        # the recovered step did advance the cells
    st.close()
    fresh.close()


def test_wait_limit_on_an_fp32_state_is_unsupported(df):
    mech, net, _, _, _ = synth.configs.build("small-fp32-4k", n_cells=8)
    st = df.State(mech, net, precision=df.DF_FP32)
    with pytest.raises(df.DFError) as e:
        st.set_wait_limit(100)
    assert e.value.code == df._lib.DF_ERR_UNSUPPORTED
    st.close()
