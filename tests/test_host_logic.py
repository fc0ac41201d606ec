"""Host-side logic that needs no GPU: the bench's guard on measured DRAM traffic, and the
autograd plumbing of ChemStepFunction (driven by a stand-in state on CPU tensors)."""
import os
import shutil

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EOS = os.path.join("paper_2508_18969_gb300", "csrc", "eos.cu")


@pytest.fixture()
def bench_copy(tmp_path, monkeypatch):
    import bench
    os.makedirs(tmp_path / os.path.dirname(EOS))
    shutil.copy(os.path.join(ROOT, EOS), tmp_path / EOS)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench, tmp_path / EOS


def test_traffic_guard_skips_only_the_other_kernels(bench_copy):
    bench, path = bench_copy
    key = ("eos_post", "32-1600-800-400-30")
    per_row = bench.MEASURED_TRAFFIC[key][2]
    assert bench.measured_traffic(*key, 1000) == pytest.approx(per_row * 1000)
    src = path.read_text()
    # an edit inside the Jacobian section keeps the figure
    marker = "// ---------------------------------------------------------------- Jacobian of the step"
    path.write_text(src.replace(marker, marker + "\n// an edited comment"))
    assert bench.measured_traffic(*key, 1000) == pytest.approx(per_row * 1000)
    # an edit of the measured kernels voids it
    path.write_text(src.replace("eos_post_kernel(EosParams P", "eos_post_kernel(EosParams  P", 1))
    assert bench.measured_traffic(*key, 1000) is None
    # so does a missing section marker
    path.write_text(src.replace(marker, "// section"))
    assert bench.measured_traffic(*key, 1000) is None


class _FakeState:
    """Stands in for State: the 'step' is T' = T + 1, Y' = 2 Y, its product g -> (3 gT, 5 gY)."""

    def __init__(self):
        self.calls = []

    def chem_step(self, T, p, Y):
        T += 1.0
        Y *= 2.0

    def chem_step_vjp(self, T, p, Y, gT, gY):
        self.calls.append((gT.clone(), gY.clone()))
        return 3.0 * gT, 5.0 * gY


def test_chem_step_function_plumbing():
    from paper_2508_18969_gb300.api import ChemStepFunction
    st = _FakeState()
    T = torch.tensor([500.0, 900.0], dtype=torch.float64, requires_grad=True)
    Y = torch.tensor([[0.25, 0.5], [0.75, 0.5]], dtype=torch.float64, requires_grad=True)
    p = torch.full((2,), 1e7, dtype=torch.float64)
    T1, Y1 = ChemStepFunction.apply(T, Y, p, st)
    assert torch.equal(T1, T.detach() + 1.0) and torch.equal(Y1, 2.0 * Y.detach())
    assert torch.equal(T.detach(), torch.tensor([500.0, 900.0], dtype=torch.float64))
    wT = torch.tensor([1.0, -2.0], dtype=torch.float64)
    wY = torch.tensor([[1.0, 2.0], [3.0, 4.0]], dtype=torch.float64)
    gT, gY = torch.autograd.grad((wT * T1).sum() + (wY * Y1).sum(), (T, Y))
    assert torch.equal(gT, 3.0 * wT) and torch.equal(gY, 5.0 * wY)
    # only Y' in the loss: T' gets a zero cotangent
    T1, Y1 = ChemStepFunction.apply(T, Y, p, st)
    (gY,) = torch.autograd.grad((wY * Y1).sum(), (Y,))
    assert torch.equal(st.calls[-1][0], torch.zeros(2, dtype=torch.float64))
    assert torch.equal(gY, 5.0 * wY)


def test_cell_arrays_are_checked_before_the_library_is_called():
    from paper_2508_18969_gb300.api import State, _check_cells
    f64 = torch.float64
    T, p, Y = torch.zeros(5, dtype=f64), torch.zeros(5, dtype=f64), torch.zeros(3, 5, dtype=f64)
    ok = dict(device_type="cpu")
    assert _check_cells(3, T, p, Y, torch.zeros(5, dtype=torch.int32),
                        torch.zeros(1, dtype=torch.int64), **ok) == 5
    assert _check_cells(3, T[:0], p[:0], Y[:, :0], **ok) == 0
    Yw = torch.zeros(3, 8, dtype=f64)[:, :5]          # a row stride above N is allowed
    assert _check_cells(3, T, p, Yw, **ok) == 5
    bad = [
        dict(T=T.float()),                             # FP32 temperatures
        dict(T=torch.zeros(10, dtype=f64)[::2]),       # strided
        dict(p=torch.zeros(4, dtype=f64)),             # wrong length
        dict(Y=torch.zeros(4, 5, dtype=f64)),          # wrong species count
        dict(Y=torch.zeros(5, 3, dtype=f64).t()),      # cells not contiguous
        dict(Y=Y.float()),
        dict(status=torch.zeros(5, dtype=torch.int64)),
        dict(status=torch.zeros(4, dtype=torch.int32)),
        dict(n_active=torch.zeros(1, dtype=torch.int32)),
    ]
    for b in bad:
        a = dict(T=T, p=p, Y=Y)
        a.update(b)
        with pytest.raises(ValueError):
            _check_cells(3, a["T"], a["p"], a["Y"], a.get("status"), a.get("n_active"), **ok)
    # a state's entry points refuse host tensors without touching the library
    st = object.__new__(State)
    st.n, st.h, st._lib, st.dt = 3, None, None, 1e-7
    from paper_2508_18969_gb300.api import Graph, active_compact_static
    O = torch.zeros(5, 3)
    for call in (lambda: st.chem_step(T, p, Y), lambda: st.chem_source(T, p, Y),
                 lambda: st.chem_jacobian(T, p, Y), lambda: st.chem_step_vjp(T, p, Y, T, Y),
                 lambda: st.real_fluid_props(T, p, Y), lambda: st.eos_pre(T, p, Y),
                 lambda: st.active_compact(T), lambda: st.eos_post(O, T, T, p, Y),
                 lambda: Graph(st, T, p, Y, None, None, None), lambda: st.train_step(T, p, Y, Y),
                 lambda: active_compact_static(T, 600.0)):
        with pytest.raises(ValueError, match="cuda"):
            call()
    # the property network's entry points, with their own argument names
    from paper_2508_18969_gb300.propnet import PropNet
    pn = object.__new__(PropNet)
    pn.n, pn.m, pn.h, pn._lib = 3, 1, None, None
    with pytest.raises(ValueError, match="^h must be on a cuda"):
        pn.infer(T, p, Y)
    with pytest.raises(ValueError, match="^h must be on a cuda"):
        pn.fit_step(T, p, Y, torch.zeros(1, 5, dtype=f64))
    assert _check_cells(1, T, None, torch.zeros(1, 5, dtype=f64), device_type="cpu",
                        names=("h", "p", "target")) == 5
    with pytest.raises(ValueError, match="^target"):
        _check_cells(1, T, None, torch.zeros(2, 5, dtype=f64), device_type="cpu",
                     names=("h", "p", "target"))
