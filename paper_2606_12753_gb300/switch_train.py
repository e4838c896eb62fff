"""Training of the learned HLL/HLLD face switch on the GPU.

The data are faces the method itself produces: runs of a periodic box (HLLD
everywhere) are paused at a few snapshots, and at each a seeded random set of
faces is sampled with ``mhd_dump_faces`` on an FP64 handle holding the
snapshot -- 16 features of the reconstructed states, and the label 1 when the
HLLD and HLL fluxes differ by more than 1e-3 in some scaled component.  The network 16 -> 32 -> 32 -> 1 is
trained with this library's BF16 tensor-core kernels (``mlp_backward``,
``mlp_adam`` on FP32 master weights); PyTorch only holds the device buffers
and draws the minibatch indices.  The threshold tau is the largest one that
keeps the recall of the label-1 class (faces that need HLLD) at or above the
target on a held-out split: every face the network is unsure about falls
back to HLLD.

This is the library's addition to the method; the paper names the two
solvers the switch chooses between (Sec. 2.2, HLLD_Solver and HLL_Solver).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import mhd
from .inputs import turbulence_3d


NPARAM = 1633


@dataclass
class FaceSet:
    X: object        # torch float32 (n, 16), device
    y: object        # torch float32 (n,), device
    snapshots: list = field(default_factory=list)   # (steps taken, faces sampled, label-1 fraction)


def he_init(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the flat parameter order W1[32][16],
    b1, W2[32][32], b2, W3[32], b3."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((32, 16)) * math.sqrt(2.0 / 16)
    w2 = rng.standard_normal((32, 32)) * math.sqrt(2.0 / 32)
    w3 = rng.standard_normal((1, 32)) * math.sqrt(2.0 / 32)
    return np.concatenate([w1.ravel(), np.zeros(32), w2.ravel(), np.zeros(32), w3.ravel(), np.zeros(1)]).astype(
        np.float32)


def collect_faces(box, nfaces: int, snapshots=(25, 50, 100, 200), seed: int = 5,
                  evolve: str = "mixed") -> FaceSet:
    """Run ``box`` with HLLD at its CFL dt (in the ``evolve`` precision) and
    sample nfaces / len(snapshots) random faces at each snapshot (total steps
    taken so far).  Features and labels always come from an FP64 handle
    holding the snapshot's state."""
    import torch
    run = mhd.Solver(box, precision=evolve, riemann="hlld")
    run.set_state(box.cell, box.face)
    lab = run if evolve == "fp64" else mhd.Solver(box, precision="fp64", riemann="hlld")
    nall = 3 * box.nx * box.ny * box.nz
    per = int(math.ceil(nfaces / len(snapshots)))
    gen = torch.Generator(device="cuda").manual_seed(seed)
    X = torch.empty((per * len(snapshots), 16), dtype=torch.float32, device="cuda")
    y = torch.empty(per * len(snapshots), dtype=torch.float32, device="cuda")
    done, info = 0, []
    for i, target in enumerate(snapshots):
        if target > done:
            run.step(-1.0, target - done)
            done = target
        if lab is not run:
            c, f = run.get_state()
            lab.set_state(c, f)
        ids = torch.randint(0, nall, (per,), device="cuda", generator=gen, dtype=torch.int64)
        xs, ys = X[i * per:(i + 1) * per], y[i * per:(i + 1) * per]
        mhd.mhd_dump_faces(lab.h, ids.data_ptr(), per, xs.data_ptr(), ys.data_ptr())
        info.append((done, per, float(ys.mean())))
    if lab is not run:
        lab.close()
    run.close()
    return FaceSet(X[:nfaces].contiguous(), y[:nfaces].contiguous(), info)


class Switch:
    """A device parameter block with its Adam moments."""

    def __init__(self, params: np.ndarray):
        import torch
        self.block = torch.zeros(mhd.mlp_param_bytes(), dtype=torch.uint8, device="cuda")
        mhd.mlp_init(self.block.data_ptr(), np.ascontiguousarray(params, dtype=np.float32))
        self.m = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
        self.g = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
        self.t = 0

    def params(self) -> np.ndarray:
        return self.block[: NPARAM * 4].view(__import__("torch").float32).cpu().numpy().copy()

    def logits(self, X):
        import torch
        z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
        mhd.mlp_forward(self.block.data_ptr(), X.data_ptr(), X.shape[0], z.data_ptr())
        return z

    def step(self, xb, yb, lr: float):
        self.g.zero_()
        mhd.mlp_backward(self.block.data_ptr(), xb.data_ptr(), yb.data_ptr(), xb.shape[0], self.g.data_ptr())
        self.t += 1
        mhd.mlp_adam(self.block.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.g.data_ptr(), self.t, lr=lr)


def bce(z, y) -> float:
    """Mean binary cross-entropy of logits z against 0/1 labels y (reporting only)."""
    import torch
    return float((torch.clamp(z, min=0) - z * y + torch.log1p(torch.exp(-torch.abs(z)))).mean())


def train(faces: FaceSet, steps: int = 3000, batch: int = 16384, lr: float = 3e-3, seed: int = 5,
          val_frac: float = 0.1):
    """Adam on random minibatches of the training split (cosine-decayed
    learning rate).  Returns the Switch and a report dict."""
    import torch
    n = faces.X.shape[0]
    gen = torch.Generator(device="cuda").manual_seed(seed + 1)
    perm = torch.randperm(n, device="cuda", generator=gen)
    nval = max(1, int(n * val_frac))
    val, tr = perm[:nval], perm[nval:]
    Xv, yv = faces.X[val].contiguous(), faces.y[val].contiguous()
    Xt, yt = faces.X[tr].contiguous(), faces.y[tr].contiguous()
    sw = Switch(he_init(seed))
    l0 = bce(sw.logits(Xv), yv)
    t0 = time.perf_counter()
    ntr = Xt.shape[0]
    # when faces that need HLLD are rare, half of every minibatch is drawn
    # from them (the threshold is then chosen on the natural distribution)
    pos = torch.nonzero(yt > 0.5).flatten()
    balance = 0 < pos.numel() < 0.25 * ntr
    for it in range(steps):
        idx = torch.randint(0, ntr, (batch,), device="cuda", generator=gen)
        if balance:
            k = torch.randint(0, pos.numel(), (batch // 2,), device="cuda", generator=gen)
            idx[: batch // 2] = pos[k]
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))
        sw.step(Xt[idx].contiguous(), yt[idx].contiguous(), max(lr_t, lr * 1e-2))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    zv = sw.logits(Xv)
    rep = {"faces": n, "train": int(ntr), "val": int(nval), "label1_frac": float(faces.y.mean()),
           "val_label1": int((yv > 0.5).sum()), "balanced_batches": bool(balance),
           "val_loss_init": l0, "val_loss": bce(zv, yv), "steps": steps, "batch": batch, "train_s": t_train}
    return sw, (Xv, yv, zv), rep


def choose_tau(zv, yv, recall: float = 0.99):
    """Largest threshold tau with recall(label 1) >= ``recall`` on the held-out
    faces, and the fraction of faces it sends to HLL."""
    import torch
    z1 = zv[yv > 0.5]
    if z1.numel() == 0:
        zt = float(zv.max()) + 1.0
    else:
        k = int(math.floor((1.0 - recall) * z1.numel()))
        zt = float(torch.sort(z1).values[k])
    zt32 = float(np.float32(zt))
    tau = 1.0 / (1.0 + math.exp(-zt32))
    tau = min(max(tau, 1e-30), 1.0 - 1e-12)
    # the kernels compare the FP32 logit with the FP32 logit of tau
    zk = float(np.float32(math.log(tau / (1.0 - tau))))
    hlld = zv >= zk
    rec = float((hlld & (yv > 0.5)).sum()) / max(int((yv > 0.5).sum()), 1)
    return tau, {"tau": tau, "logit_threshold": zk, "val_recall": rec, "val_hll_frac": float(1.0 - hlld.float().mean())}


def train_switch(n: int = 256, nfaces: int = 10_000_000, seed: int = 5, steps: int = 3000, batch: int = 16384,
                 recall: float = 0.99, snapshots=(25, 50, 100, 200), evolve: str = "mixed"):
    """The whole pipeline on a turbulence box of n^3 cells (the
    decaying-turbulence start with ``seed``): faces, training, threshold.
    Returns (Switch, tau, report)."""
    box = turbulence_3d(n, seed=seed)
    t0 = time.perf_counter()
    faces = collect_faces(box, nfaces, snapshots=snapshots, seed=seed, evolve=evolve)
    t_collect = time.perf_counter() - t0
    sw, (Xv, yv, zv), rep = train(faces, steps=steps, batch=batch, seed=seed)
    tau, trep = choose_tau(zv, yv, recall)
    rep.update(trep)
    rep.update({"box": f"turbulence {n}^3 seed {seed}", "snapshots": faces.snapshots, "collect_s": t_collect})
    return sw, tau, rep
