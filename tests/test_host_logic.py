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
