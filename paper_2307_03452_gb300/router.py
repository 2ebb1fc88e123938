"""Learned routing between the FP64 path and the split path.

A 3-layer MLP (20 -> 64 -> 64 -> 1, FP16 weights) predicts log10 of each quartet's largest
|integral| from cheap shell descriptors (lx_route_features).  The split path's absolute
error grows with the magnitude of the integrals, so quartets predicted above a threshold
tau go to the FP64 path and the rest to the split path.  Training (forward, backward,
Adam) and inference run in the library's own kernels; this module only moves tensors.
No part of the paper corresponds to it.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lx

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "router_weights.json")
FORMAT_VERSION = 1


class Router:
    def __init__(self, device="cuda", seed: int = 0):
        import torch
        self.device = device
        rng = np.random.default_rng(seed)
        p = np.zeros(lx.MLP_NPARAM, dtype=np.float32)
        nin, nw = lx.MLP_NIN, lx.MLP_WIDTH
        o = 0
        for (fan_in, n_out) in [(nin, nw), (nw, nw)]:
            p[o:o + n_out * fan_in] = rng.normal(scale=np.sqrt(2.0 / fan_in), size=n_out * fan_in)
            o += n_out * fan_in + n_out  # weights, then zero biases
        p[o:o + nw] = rng.normal(scale=np.sqrt(1.0 / nw), size=nw)
        self.params = torch.tensor(p, device=device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.p16 = self.params.half()
        self.step = 0
        self.tau = None  # routing threshold on the predicted log10 max |integral|

    # ---- inference
    def predict(self, feat):
        return lx.mlp_forward(self.p16, feat)

    # ---- training on the GPU (lx_mlp_grad + lx_mlp_adam)
    def train(self, feat, target, steps=2000, batch=4096, lr=3e-3, seed=0, log_every=0):
        import torch
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        n = feat.shape[0]
        losses = []
        for it in range(steps):
            idx = torch.randint(0, n, (min(batch, n),), device=self.device, generator=g)
            xb, tb = feat[idx].contiguous(), target[idx].contiguous()
            loss, grad = lx.mlp_grad(self.params, xb, tb)
            self.step += 1
            lr_t = lr * 0.5 * (1 + np.cos(np.pi * it / steps))  # cosine decay
            lx.mlp_adam(self.params, self.m, self.v, grad, self.p16, self.step, lr_t)
            if log_every and it % log_every == 0:
                losses.append(float(loss))
        return losses

    def loss(self, feat, target):
        loss, _ = lx.mlp_grad(self.params, feat, target)
        return float(loss)

    # ---- persistence (versioned JSON: weights, threshold, provenance)
    def save(self, path=WEIGHTS, meta=None):
        d = {"format": FORMAT_VERSION, "nin": lx.MLP_NIN, "width": lx.MLP_WIDTH,
             "params": self.params.cpu().numpy().astype(float).tolist(), "tau": self.tau, "meta": meta or {}}
        with open(path, "w") as f:
            json.dump(d, f)

    @classmethod
    def load(cls, path=WEIGHTS, device="cuda"):
        import torch
        with open(path) as f:
            d = json.load(f)
        if d.get("format") != FORMAT_VERSION or d["nin"] != lx.MLP_NIN or d["width"] != lx.MLP_WIDTH:
            raise ValueError(f"incompatible router weights file {path}")
        r = cls(device=device)
        r.params = torch.tensor(np.asarray(d["params"], dtype=np.float32), device=device)
        r.p16 = r.params.half()
        r.tau = d.get("tau")
        r.meta = d.get("meta", {})
        return r


def block_log10_max(out, off, sizes, floor=1e-300):
    """log10 of the largest |integral| of each quartet block (CUDA tensors in, CUDA tensor out)."""
    import torch
    off_t = torch.as_tensor(np.asarray(off), device=out.device)
    sz_t = torch.as_tensor(np.asarray(sizes), device=out.device)
    seg = torch.repeat_interleave(torch.arange(len(off_t), device=out.device), sz_t)
    idx = torch.repeat_interleave(off_t - torch.cumsum(sz_t, 0) + sz_t, sz_t) + torch.arange(int(sz_t.sum()),
                                                                                            device=out.device)
    vals = out[idx].abs()
    mx = torch.zeros(len(off_t), dtype=out.dtype, device=out.device).scatter_reduce(0, seg, vals, "amax")
    return torch.log10(mx.clamp_min(floor)).float()


def labels(basis, quartets, solid=True):
    """Training targets: log10 max |integral| per quartet from the FP64 path."""
    out, off = lx.eri(basis, quartets, solid=solid, path="fp64")
    b = lx.Batch(basis, quartets, solid)
    return block_log10_max(out, off, b.sizes), out, off


def routed_eri(basis, quartets, router: Router, solid=True, tau=None, device="cuda",
               workspace_limit: int = 16 << 30, return_mask: bool = True):
    """Evaluate with per-quartet routing in one library call (path "routed", after installing
    this network); returns (out, offsets, route mask: True = FP64) or (out, offsets) when
    return_mask is False.  The batch is chunked to fit workspace_limit bytes of scratch (or
    the smallest workspace that holds its largest quartet, if that is more).  The mask is
    recomputed here from the same features and network, for reporting."""
    tau = router.tau if tau is None else tau
    lx.router_set(router.p16, tau)
    out, off = lx.eri(basis, quartets, solid=solid, device=device, workspace_limit=workspace_limit, path="routed")
    if not return_mask:
        return out, off
    to_fp64 = (router.predict(lx.route_features(basis, quartets, device=device)) >= tau).cpu().numpy()
    return out, off, to_fp64 | (transform_flops(basis, quartets, solid) < ROUTE_SPLIT_MIN_FLOP)


#: quartets whose two transforms take fewer FLOPs than this go to the FP64 path (as in the library)
ROUTE_SPLIT_MIN_FLOP = 1.0e6


def transform_flops(basis, quartets, solid=True):
    """2 N_ab (K_bra N_p)(K_ket N_q) + 2 N_ab (K_ket N_q) N_cd per quartet."""
    q = np.asarray(quartets, dtype=np.int64).reshape(-1, 4)
    l, k = np.asarray(basis["l"]), np.asarray(basis["nprim"]).astype(np.float64)
    nf = (2 * l + 1) if solid else (l + 1) * (l + 2) // 2
    pyr = lambda n: (n + 1) * (n + 2) * (n + 3) / 6.0  # noqa: E731
    nab = nf[q[:, 0]] * nf[q[:, 1]] * 1.0
    ncd = nf[q[:, 2]] * nf[q[:, 3]] * 1.0
    kp = k[q[:, 0]] * k[q[:, 1]] * pyr(l[q[:, 0]] + l[q[:, 1]])
    kq = k[q[:, 2]] * k[q[:, 3]] * pyr(l[q[:, 2]] + l[q[:, 3]])
    return 2.0 * nab * kp * kq + 2.0 * nab * kq * ncd
