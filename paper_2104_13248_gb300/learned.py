"""Learned few-view correction: data generation, training and evaluation.

Pairs come from the method itself: seeded random-ellipsoid phantoms are
projected on the GPU (bp_phantom_project), the full-view FDK (all views,
FP32) is the target and the few-view FDK (every k-th view, FP16-stored
filtered projections, FP32 accumulation) the input. The U-Net is trained on
random crops of the pairs and evaluated on whole volumes of held-out seeds
against the full-view FDK; when no trained network is supplied the
reconstruction falls back to the plain full-view path.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np
import torch

from . import api, inputs
from .unet import UNet, conv_flops


def few_view_geometry(g: dict, stride: int) -> dict:
    """The same scan keeping every stride-th view (angles of views 0, stride, ...)."""
    n = g["np"]
    ang = np.asarray(g["angles"], dtype=np.float64) if g.get("angles") is not None else 2 * np.pi * np.arange(n) / n
    sel = ang[::stride]
    return inputs.scaled_geom(g, np=len(sel), angles=sel)


class PairMaker:
    """Full-view and few-view FDK of seeded phantoms, all on the GPU."""

    def __init__(self, g: dict, stride: int = 6, n_ell: int = 30, axes=(3.0, 40.0)):
        self.g = g
        self.stride = stride
        self.n_ell, self.axes = n_ell, axes
        self.full = api.bp_create(g)
        self.few = api.bp_create(few_view_geometry(g, stride))
        self.raw = torch.empty(self.full.proj_shape(), dtype=torch.float32, device="cuda")
        self.q_full = torch.empty_like(self.raw)
        nf = self.few.n_views
        self.q_few16 = torch.empty((nf, g["nv"], g["nu"]), dtype=torch.float16, device="cuda")

    def phantom(self, seed: int) -> np.ndarray:
        return inputs.random_ellipsoids(seed, self.n_ell, self.axes, self.g)

    def full_fdk(self, seed: int) -> torch.Tensor:
        api.bp_phantom_project(self.full, self.phantom(seed), out=self.raw)
        return api.fdk(self.full, self.raw, filtered=self.q_full)

    def pair(self, seed: int):
        api.bp_phantom_project(self.full, self.phantom(seed), out=self.raw)
        target = api.fdk(self.full, self.raw, filtered=self.q_full)
        raw_few = self.raw[::self.stride].contiguous()
        x = api.fdk(self.few, raw_few, out_dtype=torch.float16, filtered=self.q_few16)
        return x, target

    def close(self):
        self.full.close()
        self.few.close()


def fov_mask(g: dict, device="cuda") -> torch.Tensor:
    """Voxels inside the cylinder every view sees (0.95 x its radius)."""
    r, _ = inputs.fov_limits(g)
    x = (torch.arange(g["nx"], device=device) - 0.5 * (g["nx"] - 1)) * g["sx"]
    y = (torch.arange(g["ny"], device=device) - 0.5 * (g["ny"] - 1)) * g["sy"]
    m2 = (x[None, :] ** 2 + y[:, None] ** 2) <= (0.95 * r) ** 2
    return m2[None].expand(g["nz"], -1, -1)


def rmse(a: torch.Tensor, b: torch.Tensor, mask: torch.Tensor) -> float:
    d = (a - b)[mask].double()
    return float(torch.sqrt((d * d).mean()).item())


def make_training_set(maker: PairMaker, seeds, crop: int, crops_per_volume: int, rng: np.random.Generator):
    xs, ts = [], []
    g = maker.g
    for s in seeds:
        x, t = maker.pair(s)
        for _ in range(crops_per_volume):
            z0, y0, x0 = (int(rng.integers(0, (n - crop) // 4 + 1)) * 4 for n in (g["nz"], g["ny"], g["nx"]))
            xs.append(x[z0:z0 + crop, y0:y0 + crop, x0:x0 + crop].clone())
            ts.append(t[z0:z0 + crop, y0:y0 + crop, x0:x0 + crop].clone())
    return torch.stack(xs), torch.stack(ts)


def train(net: UNet, xs: torch.Tensor, ts: torch.Tensor, steps: int, lr: float = 1e-3, batch: int = 1,
          seed: int = 0, log_every: int = 0):
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = rng.integers(0, xs.shape[0], size=batch)
        idx_t = torch.as_tensor(idx, device=xs.device)
        lr_it = lr * 0.5 * (1 + math.cos(math.pi * it / max(1, steps)))   # cosine decay
        loss = net.train_step(xs[idx_t], ts[idx_t], lr=lr_it)
        losses.append(loss)
        if log_every and (it + 1) % log_every == 0:
            print(f"step {it + 1}: loss {np.mean(losses[-log_every:]):.5f}", flush=True)
    return losses


def evaluate(net: UNet | None, maker: PairMaker, seeds, mask: torch.Tensor):
    """RMSE vs the full-view FDK for the few-view input and (if net) its correction."""
    r_few, r_net = [], []
    for s in seeds:
        x, t = maker.pair(s)
        r_few.append(rmse(x, t, mask))
        if net is not None:
            r_net.append(rmse(net.forward(x), t, mask))
    return float(np.mean(r_few)), (float(np.mean(r_net)) if net is not None else None)


def reconstruct(maker: PairMaker, raw: torch.Tensor, net: UNet | None) -> torch.Tensor:
    """Few-view + network when a trained network is given; plain full-view FDK otherwise."""
    if net is None:
        return api.fdk(maker.full, raw, filtered=maker.q_full)
    x = api.fdk(maker.few, raw[::maker.stride].contiguous(), out_dtype=torch.float16, filtered=maker.q_few16)
    return net.forward(x)


def time_paths(maker: PairMaker, net: UNet, seed: int, reps: int = 5):
    """Wall time on the GPU of (a) full-view filter + BP and (b) few-view filter + BP + network."""
    api.bp_phantom_project(maker.full, maker.phantom(seed), out=maker.raw)
    raw_few = maker.raw[::maker.stride].contiguous()

    def tm(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_full = tm(lambda: api.fdk(maker.full, maker.raw, filtered=maker.q_full))
    t_few = tm(lambda: api.fdk(maker.few, raw_few, out_dtype=torch.float16, filtered=maker.q_few16))
    x = api.fdk(maker.few, raw_few, out_dtype=torch.float16, filtered=maker.q_few16)
    t_net = tm(lambda: net.forward(x))
    return t_full, t_few, t_net


def run(preset: str = "c5_learned", steps: int = 16000, crops_per_volume: int = 4, heldout: int | None = None,
        lr: float = 5e-4, log_every: int = 250, e1b: bool = False, d1: bool = False) -> dict:
    """The few-view workload end to end; returns a JSON-able summary."""
    p = inputs.preset(preset)
    g = p["geom"]
    maker = PairMaker(g, stride=p["geom"]["np"] // p["few"], n_ell=p["n_ell"], axes=p["axes"])
    n_vol = p["train_pairs"] // crops_per_volume
    rng = np.random.default_rng(p["seed"])
    t0 = time.time()
    xs, ts = make_training_set(maker, range(p["seed"], p["seed"] + n_vol), p["crop"], crops_per_volume, rng)
    t_data = time.time() - t0
    net = UNet(seed=p["seed"], e1b=e1b, d1=d1)
    t0 = time.time()
    losses = train(net, xs, ts, steps, lr=lr, log_every=log_every)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del xs, ts
    mask = fov_mask(g)
    n_eval = p["heldout"] if heldout is None else heldout
    seeds = range(p["heldout_seed"], p["heldout_seed"] + n_eval)
    r_few, r_net = evaluate(net, maker, seeds, mask)
    t_full, t_few, t_net = time_paths(maker, net, p["heldout_seed"])
    flops = conv_flops((1, g["nz"], g["ny"], g["nx"]), e1b=e1b, d1=d1)
    out = {"preset": preset, "train_pairs": p["train_pairs"], "crop": p["crop"], "steps": steps,
           "heldout": n_eval, "rmse_few_view": r_few, "rmse_few_view_plus_net": r_net,
           "rmse_ratio": r_net / r_few, "loss_first": float(np.mean(losses[:50])),
           "loss_last": float(np.mean(losses[-50:])), "data_s": t_data, "train_s": t_train,
           "ms_full_view_fdk": t_full, "ms_few_view_fdk": t_few, "ms_net": t_net,
           "speedup_vs_full_view": t_full / (t_few + t_net),
           "net_tflops": flops / (t_net * 1e-3) / 1e12}
    maker.close()
    return out


if __name__ == "__main__":
    import sys
    steps = int(sys.argv[1]) if len(sys.argv) > 1 else 16000
    lr = float(sys.argv[2]) if len(sys.argv) > 2 else 5e-4
    print(json.dumps(run(steps=steps, lr=lr)))
