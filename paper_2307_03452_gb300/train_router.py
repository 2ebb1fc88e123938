"""Train the router MLP on the GPU and calibrate the thresholds of its split tiers.

  python -m paper_2307_03452_gb300.train_router [--train N] [--mixed M] [--val V] [--steps S] [--out FILE]

Quartets are drawn like the routed workload (l = 4..6 per shell, K = 1..5 per shell, pair
centers within 3 bohr, bra-ket separations uniform in 0..30 bohr, exponents log-uniform in
[0.05, 50]); --mixed adds quartets like the mixed-class workload (five classes, K = 1..5,
centers in a 20-bohr cube).  Targets per quartet, from the
GPU FP64 path (itself checked against the CPU oracle by the parity tests): log10 of the
largest |integral| (output 0) and log10 of the largest |difference| between the 6-digit split
path and the FP64 path (output 1).  For each tier of 4, 5 and 6 digits the threshold is the
lowest prediction of output 1 among validation quartets whose error with that many digits
exceeds half the 1e-10 target, less a margin for the prediction error; quartets predicted at
or above every threshold take the FP64 path.  The quartets near the 4-digit tier's limit
decide its threshold and are few, so the training set holds several copies of each.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, lx
from .router import WEIGHTS, Router, block_log10_max, block_max_abs

TARGET_ABS = 1e-10
LABEL_FLOOR = -20.0  # log10 magnitudes below 1e-20 are all "tiny" for routing
WS_LIMIT = 8 << 30  # workspace per evaluation (the batch is chunked to fit)
DISABLED = -1e30  # threshold of a tier no quartet may take


def evaluate(basis, quartets, path):
    out, off = lx.eri(basis, quartets, solid=True, path=path, workspace_limit=WS_LIMIT)
    return out, off


def split_errors(basis, quartets, ref, off, sizes, path="split"):
    """Largest absolute error of each quartet on a split path, against the FP64 result ref."""
    outs, _ = evaluate(basis, quartets, path)
    return block_max_abs(outs - ref, off, sizes)


def labelled(basis, quartets, err_floor=-16.0):
    """Features, the two targets (errors below 10^err_floor are all "tiny"), and the errors of
    the 4-, 5- and 6-digit split paths."""
    import torch
    out, off = evaluate(basis, quartets, "fp64")
    sizes = lx.Batch(basis, quartets, True).sizes
    y0 = block_log10_max(out, off, sizes).clamp_min(LABEL_FLOOR)
    errs = {d: split_errors(basis, quartets, out, off, sizes, f"split{d}") for d in lx.ROUTE_TIERS}
    y1 = torch.log10(errs[6].clamp_min(1e-300)).float().clamp_min(err_floor)
    return lx.route_features(basis, quartets), torch.stack([y0, y1], dim=1).contiguous(), errs


def baseline_rmse(feat, target, feat_val, target_val):
    """RMSE of a least-squares line on the (ss|ss)-type estimate alone (feature 19)."""
    x = feat[:, 19].double().cpu().numpy() * 10.0
    y = target.double().cpu().numpy()
    A = np.column_stack([x, np.ones_like(x)])
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    xv = feat_val[:, 19].double().cpu().numpy() * 10.0
    pv = coef[0] * xv + coef[1]
    return float(np.sqrt(np.mean((pv - target_val.double().cpu().numpy()) ** 2))), coef.tolist()


def calibrate(pred_err, errs, margin):
    """Thresholds of the 4-, 5- and 6-digit tiers on the predicted log10 error (output 1)."""
    tau = []
    for d in lx.ROUTE_TIERS:
        bad = errs[d] > 0.5 * TARGET_ABS
        # no validation quartet fails this tier: its threshold is the largest prediction seen
        tau.append(float(pred_err[bad].min()) - margin if bool(bad.any()) else float(pred_err.max()) + margin)
    for i in range(1, len(tau)):  # fewer digits are never allowed more than more digits
        tau[i] = max(tau[i], tau[i - 1])
    return tau


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--train", type=int, default=200000, help="training quartets like the routed workload")
    ap.add_argument("--mixed", type=int, default=0, help="training quartets like the mixed-class workload")
    ap.add_argument("--val", type=int, default=16000, help="validation quartets of each kind")
    ap.add_argument("--steps", type=int, default=24000)
    ap.add_argument("--err-floor", type=float, default=-17.0, help="log10 floor of the error target")
    ap.add_argument("--oversample", type=int, default=8,
                    help="copies in the training set of quartets whose 4-digit error passes 1/20 of the target")
    ap.add_argument("--margin", type=float, default=0.5, help="decades between a tier's threshold and "
                                                                   "its lowest failing validation prediction")
    ap.add_argument("--seed", type=int, default=2311)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args(argv)
    torch.cuda.set_device(0)
    t0 = time.time()
    parts = [inputs.spread_distances(args.train, seed=args.seed)]
    vparts = [inputs.spread_distances(args.val, seed=args.seed + 1)]
    if args.mixed:
        parts.append(inputs.mixed_classes(args.mixed, seed=args.seed + 10))
        vparts.append(inputs.mixed_classes(args.val, seed=args.seed + 11))
    train, val = inputs.concat(parts), inputs.concat(vparts)
    ft, yt, errs_t = labelled(*train, err_floor=args.err_floor)
    fv, yv, errs = labelled(*val, err_floor=args.err_floor)
    # the quartets that decide the 4-digit threshold are few: repeat them in the training set
    hard = torch.nonzero(errs_t[4] > TARGET_ABS / 20).flatten()
    if args.oversample > 1 and len(hard):
        rep = hard.repeat(args.oversample - 1)
        ft, yt = torch.cat([ft, ft[rep]]), torch.cat([yt, yt[rep]])
    t_label = time.time() - t0
    r = Router(seed=args.seed)
    t1 = time.time()
    r.train(ft, yt, steps=args.steps, batch=4096, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    pv = r.predict(fv)
    rmse = [float(torch.sqrt(torch.mean((pv[:, o] - yv[:, o]) ** 2))) for o in range(lx.MLP_NOUT)]
    base_rmse, base_coef = baseline_rmse(ft, yt[:, 0], fv, yv[:, 0])
    near = yv[:, 1] > -14.0  # prediction error of output 1 where the thresholds live (reported)
    rmse_near = float(torch.sqrt(torch.mean((pv[near, 1] - yv[near, 1]) ** 2))) if bool(near.any()) else rmse[1]
    margin = args.margin
    r.tau = calibrate(pv[:, 1], errs, margin)
    dest = r.tiers(fv, *val)
    routed_err = torch.zeros_like(errs[6])
    for d in lx.ROUTE_TIERS:
        m = torch.as_tensor(dest == d, device=routed_err.device)
        routed_err[m] = errs[d][m]
    meta = {"train_quartets": args.train + args.mixed, "hard_quartets_repeated": int(len(hard)),
            "oversample": args.oversample, "err_floor_log10": args.err_floor,
            "val_quartets": len(vparts) * args.val, "steps": args.steps,
            "seed": args.seed, "label_source": "GPU FP64 path (output 0: log10 max |integral|, solid harmonics; "
                                               "output 1: log10 max |6-digit split - FP64|)",
            "val_rmse_log10": rmse[0], "val_rmse_log10_split_error": rmse[1],
            "val_rmse_log10_split_error_above_1e-14": rmse_near, "margin": margin,
            "label_floor_log10": LABEL_FLOOR, "baseline_rmse_log10": base_rmse, "baseline_line": base_coef,
            "split_bad_fraction_val": {str(d): float((errs[d] > 0.5 * TARGET_ABS).float().mean())
                                       for d in lx.ROUTE_TIERS},
            "tier_fraction_val": {str(d): float((dest == d).mean()) for d in (0,) + lx.ROUTE_TIERS},
            "val_routed_max_abs_err": float(routed_err.max()),
            "label_seconds": t_label, "train_seconds": t_train}
    r.save(args.out, meta)
    print(json.dumps({"tau": r.tau, **meta}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
