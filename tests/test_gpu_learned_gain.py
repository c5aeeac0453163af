"""What the trained regime network gains over the method without it.

On the 2D shear layer with its tau field: the network is trained (BF16 tensor-core
kernels) on snapshots of the plain FP64 run, then judged on a later, held-out
state of the same run:

* its predictions follow the true log10 non-equilibrium of each cell (the label the
  library computes from the true f) shortly after the training window;
* flagging the quarter of the cells it ranks closest to equilibrium changes one
  step less (L1 density difference from the plain step) than flagging the same
  number of cells at random -- the network picks the cells where the lambda -> 0
  form is a good approximation.

Runtime gain on the 512^2 workload is measured by ``bench.py --workload
shear_learned`` (see the profiles); this test checks the selection itself.
"""
import numpy as np
import pytest

from paper_1212_0204_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm, learned  # noqa: E402


def l1(a, b):
    return np.abs(a[0] - b[0]).sum() / np.abs(b[0]).sum()


def test_network_selects_near_equilibrium_cells_better_than_chance():
    case = W.shear_layer_2d(n=128, nv=32, steps=120, dv=0.4)
    X, y = learned.snapshots(case, nsnap=40, warmup=10)
    net = learned.train(X, y, epochs=6)
    assert net.val_mse < 0.1 * np.var(y)  # R^2 > 0.9 on the held-out 20 %

    # held-out state: step 55 of the same run, past the training snapshots
    # (steps 11 .. 50); the labels drift upwards with time, so much later states
    # are out of the training distribution (correlation 0.56 at step 90)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_primitive(case.rho, case.u, case.T)
    s.step(55)
    feats = s.features()
    truth = s.noneq().astype(np.float64)
    m = dvm.Mlp(dvm.BF16S)
    m.set_params(net.params)
    pred = m.forward((feats - net.shift) * net.scale).cpu().numpy().astype(np.float64)
    assert np.corrcoef(pred, truth)[0, 1] > 0.8

    blob = s.save()
    U_plain = _step_from(case, blob, None)
    nflag = case.ncells // 4
    by_net = np.zeros(case.ncells, dtype=np.uint8)
    by_net[np.argsort(pred)[:nflag]] = 1
    rng = np.random.default_rng(1212)
    errs_random = []
    for _ in range(3):
        rnd = np.zeros(case.ncells, dtype=np.uint8)
        rnd[rng.choice(case.ncells, nflag, replace=False)] = 1
        errs_random.append(l1(_step_from(case, blob, rnd), U_plain))
    err_net = l1(_step_from(case, blob, by_net), U_plain)
    assert err_net < 0.5 * min(errs_random), (err_net, errs_random)


def _step_from(case, blob, flags):
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_primitive(case.rho, case.u, case.T)
    s.load(blob)
    if flags is not None:
        s.learn_enable(dvm.LEARN_GIVEN)
        s.learn_set_flags(flags)
    s.step(1)
    U = s.moments()
    s.close()
    return U
