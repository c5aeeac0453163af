"""Training data and training of the regime network, through the C ABI.

Snapshots of the plain scheme (FP64 HOFKS on the GPU) give, per cell, the ten
regime features (``dvm_features``) and the label log10(||f - E[U]||_1 /
||E[U]||_1) (``dvm_noneq``); the network is trained on them by the library's
own kernels (``dvm_mlp_train``).  This module only sequences those calls and
moves arrays; every feature, label, forward and backward pass runs on the GPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import dvm
from . import workloads as W


@dataclass
class TrainedNet:
    params: np.ndarray       # packed FP32 parameters
    shift: np.ndarray        # input normalisation: x' = (x - shift) * scale
    scale: np.ndarray
    train_mse: float
    val_mse: float
    samples: int


def snapshots(case, nsnap: int = 200, warmup: int = 10, precision=dvm.F64):
    """Features (n, 10) and labels (n,) of nsnap consecutive states of the plain
    scheme on ``case`` after ``warmup`` steps (one snapshot per step)."""
    s = dvm.Solver.from_case(case, precision=precision)
    s.set_primitive(case.rho, case.u, case.T)
    s.step(warmup)
    X = np.empty((nsnap, case.ncells, dvm.NFEAT), dtype=np.float32)
    y = np.empty((nsnap, case.ncells), dtype=np.float32)
    for i in range(nsnap):
        s.step(1)
        X[i] = s.features()
        y[i] = s.noneq()
    s.close()
    return X.reshape(-1, dvm.NFEAT), y.reshape(-1)


def train(X, y, precision=dvm.BF16S, epochs: int = 20, batch: int = 1024, lr: float = 2e-3,
          val_frac: float = 0.2, seed: int = 1212) -> TrainedNet:
    """Adam on the mean squared error of the labels, 80/20 split by a seeded
    shuffle; inputs standardised with the training split's mean and deviation.
    BF16S: forward and backward on the tensor cores (BF16 operands, FP32
    accumulation, FP32 master weights); F32: FP32 on the CUDA cores."""
    import torch
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(y))
    nval = int(len(y) * val_frac)
    va, tr = order[:nval], order[nval:]
    shift = X[tr].mean(0)
    scale = 1.0 / np.maximum(X[tr].std(0), 1e-6)
    Xn = ((X - shift) * scale).astype(np.float32)
    Xt = torch.as_tensor(Xn[tr], device="cuda")
    yt = torch.as_tensor(y[tr], device="cuda")
    P0 = np.zeros(dvm.MLP_NPARAM, dtype=np.float32)
    # Glorot-uniform weights, zero biases (seeded)
    o = 0
    for fan_in, fan_out in ((dvm.NFEAT, dvm.MLP_HIDDEN), (dvm.MLP_HIDDEN, dvm.MLP_HIDDEN),
                            (dvm.MLP_HIDDEN, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        P0[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    P0[-1] = float(np.mean(y[tr]))
    net = dvm.Mlp(precision)
    net.set_params(P0)
    train_mse = net.train(Xt, yt, epochs=epochs, batch=batch, lr=lr, seed=seed)
    pred = net.forward(torch.as_tensor(Xn[va], device="cuda")).cpu().numpy()
    val_mse = float(np.mean((pred - y[va]) ** 2)) if nval else float("nan")
    P = net.params()
    net.close()
    return TrainedNet(P, shift.astype(np.float32), scale.astype(np.float32), float(train_mse),
                      val_mse, len(tr))


def train_for_shear_layer(n: int = 128, nv: int = 32, nsnap: int = 200, warmup: int = 10,
                          dv: float = 0.4, precision=dvm.BF16S, epochs: int = 20,
                          seed: int = W.SEED_BASE) -> TrainedNet:
    """The regime network of the 2D shear-layer workload: snapshots of the plain
    FP64 run at n x n cells (one per step after the warm-up), then training."""
    case = W.shear_layer_2d(n=n, nv=nv, steps=warmup + nsnap, dv=dv, seed=seed)
    X, y = snapshots(case, nsnap, warmup)
    return train(X, y, precision=precision, epochs=epochs, seed=seed)


def enable(solver, net: TrainedNet, thr: float, mlp_precision=dvm.BF16S, check_every: int = 10,
           check_samples: int = 1024, veto_radius: int = 2, seed: int = W.SEED_BASE):
    """Switch the learned path of ``solver`` on with the trained network."""
    solver.learn_enable(dvm.LEARN_MLP, mlp_precision=mlp_precision, thr=thr,
                        check_every=check_every, check_samples=check_samples,
                        veto_radius=veto_radius, seed=seed, shift=net.shift, scale=net.scale)
    solver.learn_set_params(net.params)
