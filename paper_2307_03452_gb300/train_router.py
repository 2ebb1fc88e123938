"""Train the router MLP on the GPU and calibrate its routing threshold.

  python -m paper_2307_03452_gb300.train_router [--train N] [--val M] [--steps S] [--out FILE]

Quartets are drawn like the routed workload (l = 4..6 per shell, K = 1..5 per shell, pair
centers within 3 bohr, bra-ket separations uniform in 0..30 bohr, exponents log-uniform in
[0.05, 50]).  Targets are log10 of each quartet's largest |integral| from the GPU FP64 path
(itself checked against the CPU oracle by the parity tests).  The threshold tau is the
largest prediction below which every validation quartet's split-path error, measured
against the FP64 path, stays under half the 1e-10 target, less a margin for prediction error.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, lx
from .router import WEIGHTS, Router, block_log10_max

TARGET_ABS = 1e-10
LABEL_FLOOR = -20.0  # log10 magnitudes below 1e-20 are all "tiny" for routing
WS_LIMIT = 8 << 30  # workspace per evaluation (the batch is chunked to fit)


def evaluate(basis, quartets, path):
    out, off = lx.eri(basis, quartets, solid=True, path=path, workspace_limit=WS_LIMIT)
    return out, off


def split_errors(basis, quartets, ref, off, sizes):
    """Largest absolute split-path error of each quartet, against the FP64 path result ref."""
    import torch
    outs, _ = evaluate(basis, quartets, "split")
    d = (outs - ref).abs()
    off_t = torch.as_tensor(off, device=d.device)
    sz_t = torch.as_tensor(np.asarray(sizes), device=d.device)
    seg = torch.repeat_interleave(torch.arange(len(off), device=d.device), sz_t)
    starts = torch.cumsum(sz_t, 0) - sz_t
    idx = torch.repeat_interleave(off_t - starts, sz_t) + torch.arange(int(sz_t.sum()), device=d.device)
    return torch.zeros(len(off), dtype=d.dtype, device=d.device).scatter_reduce(0, seg, d[idx], "amax")


def baseline_rmse(feat, target, feat_val, target_val):
    """RMSE of a least-squares line on the (ss|ss)-type estimate alone (feature 19)."""
    x = feat[:, 19].double().cpu().numpy() * 10.0
    y = target.double().cpu().numpy()
    A = np.column_stack([x, np.ones_like(x)])
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    xv = feat_val[:, 19].double().cpu().numpy() * 10.0
    pv = coef[0] * xv + coef[1]
    return float(np.sqrt(np.mean((pv - target_val.double().cpu().numpy()) ** 2))), coef.tolist()


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--train", type=int, default=24000)
    ap.add_argument("--val", type=int, default=4000)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--seed", type=int, default=2311)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    bt, qt = inputs.spread_distances(args.train, seed=args.seed)
    bv, qv = inputs.spread_distances(args.val, seed=args.seed + 1)
    out_t, off_t = evaluate(bt, qt, "fp64")
    yt = block_log10_max(out_t, off_t, lx.Batch(bt, qt, True).sizes).clamp_min(LABEL_FLOOR)
    del out_t
    out_v, off_v = evaluate(bv, qv, "fp64")
    sizes_v = lx.Batch(bv, qv, True).sizes
    yv = block_log10_max(out_v, off_v, sizes_v).clamp_min(LABEL_FLOOR)
    t_label = time.time() - t0
    ft = lx.route_features(bt, qt)
    fv = lx.route_features(bv, qv)
    r = Router(seed=args.seed)
    t1 = time.time()
    r.train(ft, yt, steps=args.steps, batch=4096, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    pv = r.predict(fv)
    rmse = float(torch.sqrt(torch.mean((pv - yv) ** 2)))
    base_rmse, base_coef = baseline_rmse(ft, yt, fv, yv)
    # threshold: quartets whose split error exceeds half the target must be predicted >= tau
    err_v = split_errors(bv, qv, out_v, off_v, sizes_v)
    bad = err_v > 0.5 * TARGET_ABS
    near = yv > -8.0  # prediction error where the threshold lives
    rmse_near = float(torch.sqrt(torch.mean((pv[near] - yv[near]) ** 2))) if bool(near.any()) else rmse
    margin = max(0.5, 1.5 * rmse_near)
    if bool(bad.any()):
        tau = float(pv[bad].min()) - margin
    else:
        tau = float(pv.max()) + 1.0
    r.tau = tau
    routed_fp64 = float((pv >= tau).float().mean())
    routed_ok = bool((err_v[pv < tau] <= TARGET_ABS).all()) if bool((pv < tau).any()) else True
    meta = {"train_quartets": args.train, "val_quartets": args.val, "steps": args.steps, "seed": args.seed,
            "label_source": "GPU FP64 path, log10 max |integral| (solid harmonics)",
            "val_rmse_log10": rmse, "val_rmse_log10_above_1e-8": rmse_near, "margin": margin,
            "label_floor_log10": LABEL_FLOOR, "baseline_rmse_log10": base_rmse, "baseline_line": base_coef,
            "split_bad_fraction_val": float(bad.float().mean()), "fp64_fraction_val": routed_fp64,
            "val_routed_within_target": routed_ok, "label_seconds": t_label, "train_seconds": t_train}
    r.save(args.out, meta)
    print(json.dumps({"tau": tau, **meta}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
