"""The learned router: features, the MLP's forward pass and gradient against the CPU
reference (oracle/mlp.py), training on the GPU, and what routing gains: every quartet within the
1e-10 target at fewer digit products than any single digit count that meets it."""
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
    t = rng.normal(size=(n, omlp.NOUT)).astype(np.float32)
    return p, X, t


@pytest.mark.parametrize("n", [1, 77, 1000])
def test_mlp_forward_and_gradient_match_oracle(n):
    p, X, t = _random_problem(n, n)
    p16 = p.astype(np.float16).astype(np.float64)  # the GPU forward uses FP16 weights
    pt = torch.tensor(p, device="cuda")
    Xt, tt = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    y = lx.mlp_forward(pt.half(), Xt).cpu().numpy()
    yref, _ = omlp.forward(p16, X.astype(np.float64))
    assert y.shape == (n, omlp.NOUT)
    assert np.allclose(y, yref, rtol=1e-4, atol=1e-4)
    loss, grad = lx.mlp_grad(pt, Xt, tt)
    lref, gref = omlp.loss_and_grad(p16, X.astype(np.float64), t.astype(np.float64))
    assert float(loss) == pytest.approx(lref, rel=1e-4)
    g = grad.cpu().numpy()
    assert np.allclose(g, gref, rtol=2e-3, atol=2e-5 * np.abs(gref).max())


def test_training_reduces_loss():
    # smooth synthetic targets of the features, one per output: the loss must fall by a large factor
    rng = np.random.default_rng(3)
    X = rng.normal(size=(8192, omlp.NIN)).astype(np.float32)
    t = np.stack([np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 19], np.cos(X[:, 3]) - 0.3 * X[:, 4]],
                 axis=1).astype(np.float32)
    Xt, tt = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    r = rt.Router(seed=1)
    before = r.loss(Xt, tt)
    r.train(Xt, tt, steps=600, batch=2048, lr=3e-3)
    after = r.loss(Xt, tt)
    assert after < 0.1 * before, (before, after)


needs_weights = pytest.mark.skipif(not os.path.exists(rt.WEIGHTS), reason="no trained router weights")


def _block_errors(a, b, off, sizes):
    return rt.block_max_abs(a - b, off, sizes).cpu().numpy()


@needs_weights
def test_magnitude_prediction_beats_the_physics_estimate():
    # output 0 on held-out quartets of the routed workload's distribution (a seed the training
    # never saw): closer to log10 max |integral| than a least-squares line on the (ss|ss)-type
    # estimate the network is given
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(600, seed=777, kmax=3)
    ref, off = lx.eri(basis, quartets, solid=True, path="fp64")
    sizes = lx.Batch(basis, quartets, True).sizes
    y = rt.block_log10_max(ref, off, sizes).clamp_min(r.meta.get("label_floor_log10", -20.0))
    feat = lx.route_features(basis, quartets)
    pred = r.predict(feat)[:, 0]
    rmse = float(torch.sqrt(torch.mean((pred - y) ** 2)))
    line = r.meta["baseline_line"]
    base = line[0] * feat[:, 19].double() * 10 + line[1]
    base_rmse = float(torch.sqrt(torch.mean((base.float() - y) ** 2)))
    assert rmse < base_rmse, (rmse, base_rmse)


@needs_weights
def test_routing_gain_fails_without_the_network():
    # Held-out quartets of the routed workload's distribution (l = 4..6, K = 1..5, separations
    # 0..30 bohr; a seed neither training nor validation used).  Without the network there are
    # two choices: one digit count for every quartet, where 4 digits miss the 1e-10 target and 5
    # cost 15 digit products per quartet, or the FP64 path, 20 times slower.  The routed call
    # must keep every quartet within the target at fewer digit products than 5 digits everywhere,
    # sending few quartets to the FP64 path.
    r = rt.Router.load()
    basis, quartets = inputs.routed(nquartet=8000, seed=2413)
    ref, off = lx.eri(basis, quartets, solid=True, path="fp64", workspace_limit=32 << 30)
    sizes = lx.Batch(basis, quartets, True).sizes
    split4, _ = lx.eri(basis, quartets, solid=True, path="split4", workspace_limit=32 << 30)
    e4 = _block_errors(split4, ref, off, sizes)
    del split4
    assert e4.max() > 1e-10, "4 digits everywhere meet the target: this set shows no gain"
    routed, roff, dest = rt.routed_eri(basis, quartets, r, workspace_limit=32 << 30)
    assert np.array_equal(roff, off)
    er = _block_errors(routed, ref, off, sizes)
    assert er.max() <= 1e-10, f"routed error {er.max():.3e}"
    assert np.all(dest[e4 > 0.5e-10] != 4)  # the quartets 4 digits cannot carry are moved up
    frac = {d: float(np.mean(dest == d)) for d in (0, 4, 5, 6)}
    products = sum(frac[d] * d * (d + 1) / 2 for d in (4, 5, 6))  # digit products per quartet
    assert frac[0] < 0.05, frac
    assert products < 0.9 * 15, frac


@needs_weights
def test_routed_result_against_cpu_oracle():
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(24, seed=778, kmin=1, kmax=2)
    routed, off, _ = rt.routed_eri(basis, quartets, r)
    ref, roff = oracle.eri(basis, quartets, solid=True)
    assert np.abs(routed.cpu().numpy() - ref).max() <= 1e-10


@needs_weights
def test_routed_library_call_partitions_exactly():
    # one "routed" call = the FP64 path on the quartets sent there plus each split tier on its
    # quartets, bit for bit; thresholds far above or below every prediction give one path alone
    r = rt.Router.load()
    basis, quartets = inputs.spread_distances(300, seed=779, kmax=2)
    qs = np.asarray(quartets, dtype=np.int32)
    a64, off = lx.eri(basis, qs, solid=True, path="fp64")
    a4, _ = lx.eri(basis, qs, solid=True, path="split4")
    big = rt.transform_flops(basis, qs) >= rt.ROUTE_SPLIT_MIN_FLOP
    for tau, ref in (([1e30] * 3, a4), ([-1e30] * 3, a64)):
        lx.router_set(r.p16, tau)
        got, goff = lx.eri(basis, qs, solid=True, path="routed")
        assert np.array_equal(goff, off)
        if ref is a4:  # quartets below the size rule take the FP64 path regardless
            mask = torch.as_tensor(np.repeat(big, lx.Batch(basis, qs, True).sizes), device="cuda")
            ref = torch.where(mask, a4, a64)
        assert torch.equal(got, ref)
    err = r.predict(lx.route_features(basis, qs))[:, 1].cpu().numpy()
    tau = [float(np.quantile(err, 0.25)), float(np.quantile(err, 0.5)), float(np.quantile(err, 0.75))]
    got, _, dest = rt.routed_eri(basis, qs, r, tau=tau)
    assert len(set(dest.tolist())) == 4  # every destination is used
    comp = torch.zeros_like(got)
    for d, path in ((0, "fp64"), (4, "split4"), (5, "split5"), (6, "split")):
        m = dest == d
        b = lx.Batch(basis, qs[m], True, out_off=off[m], path=path)
        b.run(comp, lx.alloc_workspace(b.workspace_size()))
    torch.cuda.synchronize()
    assert torch.equal(got, comp)


@needs_weights
def test_routed_small_quartets_take_the_fp64_path():
    # (dd|dd) at K = 1 is below the split path's break-even size: with thresholds that send
    # every prediction to the 4-digit tier, routing still sends these quartets to the FP64
    # path, while the (gg|gg) quartets beside them take the split path
    r = rt.Router.load()
    small = inputs.uniform_class((2, 2, 2, 2), 6, 780, cube=4.0, exps=(0.1, 10.0))
    big = inputs.uniform_class((4, 4, 4, 4), 3, 781, cube=4.0, exps=(0.1, 10.0))
    basis, qs = inputs.concat([small, big])
    qs = np.asarray(qs, dtype=np.int32)
    assert np.all(rt.transform_flops(basis, qs[:6]) < rt.ROUTE_SPLIT_MIN_FLOP)
    assert np.all(rt.transform_flops(basis, qs[6:]) >= rt.ROUTE_SPLIT_MIN_FLOP)
    a64, off = lx.eri(basis, qs, solid=True, path="fp64")
    a4, _ = lx.eri(basis, qs, solid=True, path="split4")
    lx.router_set(r.p16, [1e30] * 3)
    got, _ = lx.eri(basis, qs, solid=True, path="routed")
    n_small = int(off[6])
    assert torch.equal(got[:n_small], a64[:n_small])
    assert torch.equal(got[n_small:], a4[n_small:])
