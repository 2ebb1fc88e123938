"""Learned routing between the FP64 path and the split path's digit tiers.

A 3-layer MLP (20 -> 64 -> 64 -> 2, FP16 weights) predicts, from cheap shell descriptors
(lx_route_features), log10 of each quartet's largest |integral| (output 0) and log10 of the
split path's absolute error on it with 6 digits (output 1).  That error follows the size of
the quartet's intermediates, which exceeds the result by orders of magnitude when the
Hermite sums cancel, so routing uses output 1: a quartet takes the split path with the
fewest digits (4, 5 or 6) whose threshold lies above its prediction, and the FP64 path if
none does.  Training (forward, backward, Adam) and inference run in the library's own
kernels; this module only moves tensors.  No part of the paper corresponds to it.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lx

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "router_weights.json")
FORMAT_VERSION = 2


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
        p[o:o + lx.MLP_NOUT * nw] = rng.normal(scale=np.sqrt(1.0 / nw), size=lx.MLP_NOUT * nw)
        self.params = torch.tensor(p, device=device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.p16 = self.params.half()
        self.step = 0
        self.tau = None  # thresholds of the 4-, 5- and 6-digit tiers on the predicted log10 split error

    # ---- inference
    def predict(self, feat):
        """(n, 2): predicted log10 max |integral| and log10 split error (6 digits)."""
        return lx.mlp_forward(self.p16, feat)

    def tiers(self, feat, basis=None, quartets=None, solid=True):
        """Destination of each quartet as the library routes it: 0 = FP64 path, 4, 5, 6 = the
        split path with that many digits (numpy int array)."""
        err = self.predict(feat)[:, 1].cpu().numpy()
        dest = np.zeros(len(err), dtype=np.int64)
        undecided = np.ones(len(err), dtype=bool)
        for d, t in zip(lx.ROUTE_TIERS, self.tau):
            take = undecided & (err < t)
            dest[take] = d
            undecided &= ~take
        if basis is not None:
            dest[transform_flops(basis, quartets, solid) < ROUTE_SPLIT_MIN_FLOP] = 0
        return dest

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
        d = {"format": FORMAT_VERSION, "nin": lx.MLP_NIN, "width": lx.MLP_WIDTH, "nout": lx.MLP_NOUT,
             "params": self.params.cpu().numpy().astype(float).tolist(), "tau": list(self.tau), "meta": meta or {}}
        with open(path, "w") as f:
            json.dump(d, f)

    @classmethod
    def load(cls, path=WEIGHTS, device="cuda"):
        import torch
        with open(path) as f:
            d = json.load(f)
        if (d.get("format") != FORMAT_VERSION or d["nin"] != lx.MLP_NIN or d["width"] != lx.MLP_WIDTH
                or d.get("nout") != lx.MLP_NOUT):
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
    return torch.log10(block_max_abs(out, off, sizes).clamp_min(floor)).float()


def block_max_abs(x, off, sizes):
    """Largest |x| of each quartet block (CUDA tensors in, CUDA tensor out)."""
    import torch
    off_t = torch.as_tensor(np.asarray(off), device=x.device)
    sz_t = torch.as_tensor(np.asarray(sizes), device=x.device)
    seg = torch.repeat_interleave(torch.arange(len(off_t), device=x.device), sz_t)
    idx = torch.repeat_interleave(off_t - torch.cumsum(sz_t, 0) + sz_t, sz_t) + torch.arange(int(sz_t.sum()),
                                                                                            device=x.device)
    return torch.zeros(len(off_t), dtype=x.dtype, device=x.device).scatter_reduce(0, seg, x[idx].abs(), "amax")


def routed_eri(basis, quartets, router: Router, solid=True, tau=None, device="cuda",
               workspace_limit: int = 16 << 30, return_tiers: bool = True):
    """Evaluate with per-quartet routing in one library call (path "routed", after installing
    this network and its thresholds); returns (out, offsets, destination per quartet: 0 =
    FP64, else the digits of its split tier) or (out, offsets) when return_tiers is False.
    The batch is chunked to fit workspace_limit bytes of scratch (or the smallest workspace
    that holds its largest quartet, if that is more).  The destinations are recomputed here
    from the same features, network and thresholds, for reporting."""
    tau = router.tau if tau is None else tau
    lx.router_set(router.p16, tau)
    out, off = lx.eri(basis, quartets, solid=solid, device=device, workspace_limit=workspace_limit, path="routed")
    if not return_tiers:
        return out, off
    saved, router.tau = router.tau, tau
    dest = router.tiers(lx.route_features(basis, quartets, device=device), basis, quartets, solid)
    router.tau = saved
    return out, off, dest


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
