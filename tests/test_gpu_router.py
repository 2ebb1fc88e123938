"""The learned router: features, the MLP's forward pass and gradient against the CPU
reference (oracle/mlp.py), training on the GPU, and what routing gains."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2307_03452_gb300 import inputs, lx
from paper_2307_03452_gb300 import router as rt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.set_device(0)


def test_features_follow_their_definition():
    basis, quartets = inputs.spread_distances(50, seed=5)
    f = lx.route_features(basis, quartets).cpu().numpy()
    for i, q in enumerate(quartets):
        zmin = [basis["exps"][basis["prim_off"][s]:basis["prim_off"][s] + basis["nprim"][s]].min() for s in q]
        zmax = [basis["exps"][basis["prim_off"][s]:basis["prim_off"][s] + basis["nprim"][s]].max() for s in q]
        c = basis["center"][q]
        zp, zq = zmin[0] + zmin[1], zmin[2] + zmin[3]
        P = (zmin[0] * c[0] + zmin[1] * c[1]) / zp
        Q = (zmin[2] * c[2] + zmin[3] * c[3]) / zq
        ab2, cd2, pq2 = np.sum((c[0] - c[1]) ** 2), np.sum((c[2] - c[3]) ** 2), np.sum((P - Q) ** 2)
        ref = np.zeros(20)
        ref[0:4] = basis["l"][q] / 6
        ref[4:8] = np.log(zmin) / 4
        ref[8:12] = np.log(zmax) / 4
        ref[12], ref[13], ref[14] = math.sqrt(ab2) / 10, math.sqrt(cd2) / 10, math.sqrt(pq2) / 30
        mu, nu, rho = zmin[0] * zmin[1] / zp, zmin[2] * zmin[3] / zq, zp * zq / (zp + zq)
        ref[15], ref[16] = min(mu * ab2 / 20, 10), min(nu * cd2 / 20, 10)
        T = rho * pq2
        ref[17] = math.log1p(T) / 3
        ref[18] = math.log(np.prod(basis["nprim"][q])) / 6
        f0 = 1.0 if T < 1e-6 else min(1.0, math.sqrt(math.pi / (4 * T)))
        lest = math.log(2 * math.pi ** 2.5 / (zp * zq * math.sqrt(zp + zq))) - mu * ab2 - nu * cd2 + math.log(f0)
        ref[19] = max(lest / math.log(10) / 10, -10)
        assert np.allclose(f[i], ref, rtol=2e-5, atol=2e-5), i


def _random_problem(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(scale=0.25, size=omlp.NPARAM).astype(np.float32)
    X = rng.normal(size=(n, omlp.NIN)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    return p, X, t


@pytest.mark.parametrize("n", [1, 77, 1000])
def test_mlp_forward_and_gradient_match_oracle(n):
    p, X, t = _random_problem(n, n)
    p16 = p.astype(np.float16).astype(np.float64)  # the GPU forward uses FP16 weights
    pt = torch.tensor(p, device="cuda")
    Xt, tt = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    y = lx.mlp_forward(pt.half(), Xt).cpu().numpy()
    yref, _ = omlp.forward(p16, X.astype(np.float64))
    assert np.allclose(y, yref, rtol=1e-4, atol=1e-4)
    loss, grad = lx.mlp_grad(pt, Xt, tt)
    lref, gref = omlp.loss_and_grad(p16, X.astype(np.float64), t.astype(np.float64))
    assert float(loss) == pytest.approx(lref, rel=1e-4)
    g = grad.cpu().numpy()
    assert np.allclose(g, gref, rtol=2e-3, atol=2e-5 * np.abs(gref).max())


def test_training_reduces_loss():
    # a smooth synthetic target of the features: the loss must fall by a large factor
    rng = np.random.default_rng(3)
    X = rng.normal(size=(8192, omlp.NIN)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 19]).astype(np.float32)
    Xt, tt = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    r = rt.Router(seed=1)
    before = r.loss(Xt, tt)
    r.train(Xt, tt, steps=600, batch=2048, lr=3e-3)
    after = r.loss(Xt, tt)
    assert after < 0.1 * before, (before, after)


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_routing_gain_on_held_out_quartets():
    # held-out quartets of the routed workload's distribution (a seed the training never saw)
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(600, seed=777, kmax=3)
    ref, off = lx.eri(basis, quartets, solid=True, path="fp64")
    sizes = lx.Batch(basis, quartets, True).sizes
    routed, roff, to_fp64 = rt.routed_eri(basis, quartets, r)
    assert np.array_equal(off, roff)
    err_routed = float((routed - ref).abs().max())
    assert err_routed <= 1e-10, err_routed
    # the network's magnitude prediction beats the one-feature physics estimate it is given
    y = rt.block_log10_max(ref, off, sizes).clamp_min(r.meta.get("label_floor_log10", -20.0))
    pred = r.predict(lx.route_features(basis, quartets))
    rmse = float(torch.sqrt(torch.mean((pred - y) ** 2)))
    line = r.meta["baseline_line"]
    base = line[0] * lx.route_features(basis, quartets)[:, 19].double() * 10 + line[1]
    base_rmse = float(torch.sqrt(torch.mean((base.float() - y) ** 2)))
    assert rmse < base_rmse, (rmse, base_rmse)
    # most quartets take the fast path
    assert to_fp64.mean() < 0.5


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_routed_result_against_cpu_oracle():
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(24, seed=778, kmin=1, kmax=2)
    routed, off, _ = rt.routed_eri(basis, quartets, r)
    ref, roff = oracle.eri(basis, quartets, solid=True)
    assert np.abs(routed.cpu().numpy() - ref).max() <= 1e-10


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_routed_library_call_partitions_exactly():
    # one "routed" call = the FP64 path on the quartets predicted >= tau plus the split path on
    # the rest, bit for bit; tau far above or below every prediction gives one path alone
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(300, seed=779, kmax=2)
    qs = np.asarray(quartets, dtype=np.int32)
    a64, off = lx.eri(basis, qs, solid=True, path="fp64")
    asp, _ = lx.eri(basis, qs, solid=True, path="split")
    for tau, ref in ((1e30, asp), (-1e30, a64)):
        lx.router_set(r.p16, tau)
        got, goff = lx.eri(basis, qs, solid=True, path="routed")
        assert np.array_equal(goff, off)
        assert torch.equal(got, ref)
    pred = r.predict(lx.route_features(basis, qs)).cpu().numpy()
    tau = float(np.median(pred))  # about half each way
    lx.router_set(r.p16, tau)
    got, _ = lx.eri(basis, qs, solid=True, path="routed")
    mask = (pred >= tau) | (rt.transform_flops(basis, qs) < rt.ROUTE_SPLIT_MIN_FLOP)
    assert 0 < mask.sum() < len(mask)
    comp = torch.zeros_like(got)
    for m, path in ((mask, "fp64"), (~mask, "split")):
        b = lx.Batch(basis, qs[m], True, out_off=off[m], path=path)
        b.run(comp, lx.alloc_workspace(b.workspace_size()))
    torch.cuda.synchronize()
    assert torch.equal(got, comp)


@pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")
def test_routed_small_quartets_take_the_fp64_path():
    # (dd|dd) at K = 1 is below the split path's break-even size: with the threshold set so that
    # every prediction says "split", routing still sends these quartets to the FP64 path, while
    # the (gg|gg) quartets beside them take the split path
    r = rt.Router.load()
    small = inputs.uniform_class((2, 2, 2, 2), 6, 780, cube=4.0, exps=(0.1, 10.0))
    big = inputs.uniform_class((4, 4, 4, 4), 3, 781, cube=4.0, exps=(0.1, 10.0))
    basis, qs = inputs.concat([small, big])
    qs = np.asarray(qs, dtype=np.int32)
    assert np.all(rt.transform_flops(basis, qs[:6]) < rt.ROUTE_SPLIT_MIN_FLOP)
    assert np.all(rt.transform_flops(basis, qs[6:]) >= rt.ROUTE_SPLIT_MIN_FLOP)
    a64, off = lx.eri(basis, qs, solid=True, path="fp64")
    asp, _ = lx.eri(basis, qs, solid=True, path="split")
    lx.router_set(r.p16, 1e30)
    got, _ = lx.eri(basis, qs, solid=True, path="routed")
    n_small = int(off[6])
    assert torch.equal(got[:n_small], a64[:n_small])
    assert torch.equal(got[n_small:], asp[n_small:])
