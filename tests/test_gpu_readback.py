"""Pipelined read-back of the moments (dvm_moments_async / dvm_moments_wait).

* every step's moments read back while later steps run equal, bit for bit, the
  moments of the same run read synchronously after each step (FP32 windowed 2D and
  FP64 1D), with three read-backs in flight (the slot reuse waits on the device),
  into pinned host tensors, numpy arrays and CUDA tensors;
* the status word travels with the snapshot: the 50^2 vortex with FKS on the
  coarse 20^2 velocity grid leaves the physical states at step 7, and exactly the
  read-backs from step 7 on report DVM_ERR_NONPHYSICAL;
* the batch read-back (dvm_batch_moments_async / _wait) of 16 uneven tubes equals
  the synchronous dvm_batch_moments of the same run, bit for bit;
* a ticket that was never issued is rejected.
"""
import numpy as np
import pytest

from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm  # noqa: E402


def solver(case, precision, scheme=None):
    s = dvm.Solver.from_case(case, precision=precision, scheme=scheme)
    s.set_moments(conserved(case))
    return s


@pytest.mark.parametrize("which", ["quadrant_f32", "sod_f64"])
def test_pipelined_readback_equals_synchronous(which):
    if which == "quadrant_f32":
        case, prec = W.quadrant_2d(n=64, nv=16, tau=1e-3, steps=6, dv=0.7), dvm.F32
    else:
        case, prec = W.sod_1d(nx=200, nv=32, tau=1e-4), dvm.F64
    steps = 7
    ref = solver(case, prec)
    want = []
    for _ in range(steps):
        ref.step(1)
        want.append(ref.moments())
    ref.close()

    s = solver(case, prec)
    shape = (case.d + 2, case.ncells)
    bufs = [torch.empty(shape, dtype=torch.float64).pin_memory(), np.empty(shape),
            torch.empty(shape, dtype=torch.float64, device="cuda")]
    got, tickets = [], []
    for i in range(steps):
        s.step_async(1)
        tickets.append(s.moments_async(bufs[i % 3]))
        if i >= 2:  # three in flight, then read the oldest
            s.moments_wait(tickets[i - 2])
            b = bufs[(i - 2) % 3]
            got.append(b.cpu().numpy().copy() if isinstance(b, torch.Tensor) else b.copy())
    for i in range(steps - 2, steps):
        s.moments_wait(tickets[i])
        b = bufs[i % 3]
        got.append(b.cpu().numpy().copy() if isinstance(b, torch.Tensor) else b.copy())
    assert tickets == list(range(steps))
    s.close()
    for i in range(steps):
        assert np.array_equal(got[i], want[i]), i


def test_readback_carries_the_status_of_its_step():
    case = W.isentropic_vortex_2d(50, nv=20, vmax=15.0, t_final=8 * 0.2 / 1.5, scheme=W.FKS)
    s = solver(case, dvm.F64, scheme=dvm.FKS)
    out = [np.empty((4, case.ncells)) for _ in range(case.steps)]
    tickets = []
    for i in range(case.steps):
        s.step_async(1)
        tickets.append(s.moments_async(out[i]))
    for i in range(6):
        s.moments_wait(tickets[i])
        assert out[i][0].min() > 0
    with pytest.raises(dvm.DvmError) as e:
        s.moments_wait(tickets[6])
    assert e.value.code == -5
    s.close()


def test_unissued_ticket_is_rejected():
    case = W.sod_1d(nx=50, nv=16, tau=1e-4)
    s = solver(case, dvm.F64)
    s.step(1)
    with pytest.raises(dvm.DvmError) as e:
        s.moments_wait(0)
    assert e.value.code == -1
    s.close()


def test_batch_pipelined_readback_equals_synchronous():
    cases = W.batched_tubes(ncases=16, steps=5, nx_range=(40, 300))
    U0 = None
    want = []
    b = dvm.Batch(cases, precision=dvm.F32)
    U0 = b.pack([conserved(c) for c in cases])
    b.set_moments(U0)
    for _ in range(5):
        b.step(1)
        want.append(b.moments())
    b.close()
    b = dvm.Batch(cases, precision=dvm.F32)
    b.set_moments(U0)
    bufs = [torch.empty((3, b.ncells), dtype=torch.float64).pin_memory() for _ in range(2)]
    got, prev = [], None
    for i in range(5):
        b.step_async(1)
        t = b.moments_async(bufs[i & 1])
        if prev is not None:
            b.moments_wait(prev)
            got.append(bufs[(i - 1) & 1].numpy().copy())
        prev = t
    b.moments_wait(prev)
    got.append(bufs[4 & 1].numpy().copy())
    b.close()
    for i in range(5):
        assert np.array_equal(got[i], want[i]), i
