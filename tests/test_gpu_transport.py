"""Parity of df_transport_props (Chung et al. 1988 at the Peng-Robinson density) with the FP64
transport oracle, through the C ABI. The Peng-Robinson state and the outer mixing sums are FP64
on the GPU; the FP32 inner pair sums and the FP32 evaluation of the correlation leave differences
of up to 1e-5 relative (measured on GB300: mu 9.8e-6, lambda and alpha 2.7e-6); the bound is ten
times that."""
import numpy as np
import pytest

import synth
from oracle import transport as otr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
RTOL = 1e-4


@pytest.fixture(scope="module")
def df():
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as m
    return m


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


@pytest.mark.parametrize("name,N", [("small-fp32-4k", 4096), ("layer1d-30sp-1m", 6000),
                                    ("train30-1m", 6000), ("mix3d-30sp-64m", 3000)])
def test_transport_props_vs_oracle(df, name, N):
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N)
    st = df.State(mech, net, batch_cells=1024)
    mu, lam, alpha = (a.cpu().numpy() for a in st.transport_props(_dev(T), _dev(p), _dev(Y)))
    o = otr.state(mech, T, p, Y)
    ok = o["status"] == 0
    assert np.all(np.isnan(mu[~ok]))
    rel = {k: np.abs(g[ok] / o[k][ok] - 1.0).max() for k, g in (("mu", mu), ("lam", lam), ("alpha", alpha))}
    print(f"ERR transport {name}: " + " ".join(f"{k} rel {v:.3e}" for k, v in rel.items()))
    for k, v in rel.items():
        assert v <= RTOL, (k, v)
    st.close()


def test_transport_props_pure_fluid_nonfinite_cells_and_null_outputs(df):
    from test_gpu_parity import _extreme_case
    mech, net, T, p, Y = _extreme_case(1, 700, 41)
    T = T.copy()
    p = p.copy()
    T[3] = np.nan
    p[5] = -1.0
    st = df.State(mech, net, precision=df.DF_FP32, T_react=0.0, batch_cells=1024)
    mu, lam, alpha = (a.cpu().numpy() for a in st.transport_props(_dev(T), _dev(p), _dev(Y)))
    good = np.ones(T.shape[0], bool)
    good[[3, 5]] = False
    assert np.all(np.isnan(mu[~good])) and np.all(np.isnan(alpha[~good]))
    o = otr.state(mech, T[good], p[good], Y[:, good])
    np.testing.assert_allclose(mu[good], o["mu"], rtol=RTOL)
    np.testing.assert_allclose(lam[good], o["lam"], rtol=RTOL)
    # outputs may be NULL
    lib = df._lib.load()
    import ctypes
    Td, pd, Yd = _dev(T), _dev(p), _dev(Y)
    out = torch.full((T.shape[0],), -1.0, dtype=torch.float64, device=DEV)
    rc = lib.df_transport_props(st.h, T.shape[0], ctypes.c_void_p(Td.data_ptr()),
                                ctypes.c_void_p(pd.data_ptr()), ctypes.c_void_p(Yd.data_ptr()),
                                Yd.stride(0), None, ctypes.c_void_p(out.data_ptr()), None, None)
    torch.cuda.synchronize()
    assert rc == 0
    np.testing.assert_array_equal(out.cpu().numpy(), lam)
    st.close()
