"""Learned boundary upsampler on the GPU against the FP64 oracle
(oracle/mlp.py), through the C ABI: features, targets, the fused bf16
tensor-core forward, the backward pass, training, and its use inside the
lattice Boltzmann step."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from gpucases import Case, GpuRunner, interior, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = 16
U_MAX = 0.05


@pytest.fixture(scope="module")
def lbt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0809_4958_gb300 import lbtracer
    lbtracer.load()
    return lbtracer


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def master_vector(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]]).astype(np.float32)


def split_master(v, K):
    sizes = [("W1", (32, 128)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 3 * K)), ("b3", (3 * K,))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = np.asarray(v[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def bf16_params(p):
    """The parameters the GPU forward uses: weights rounded to bf16, biases f32."""
    q = {k: v.copy() for k, v in p.items()}
    for k in ("W1", "W2", "W3"):
        q[k] = bf16(q[k])
    for k in ("b1", "b2", "b3"):
        q[k] = np.asarray(q[k], np.float32).astype(np.float64)
    return q


@pytest.fixture(scope="module")
def data():
    from paper_0809_4958_gb300 import inputs
    E = 16
    modes = inputs.mode_table(21, 128, 1.0, 8.0, E)
    fine = oracle.face_samples(modes, E, 1, 0, 5 * K + 1)  # every step
    coarse = fine[::K]
    return E, fine, coarse


def test_features_and_targets_match_oracle(lbt, data):
    E, fine, coarse = data
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    for j in (0, 1, 2):
        X = lbt.mlp_features(d(coarse[max(j - 1, 0)]), d(coarse[j]), d(coarse[j + 1]), d(coarse[j + 2]), E, U_MAX)
        X = X.float().cpu().numpy().astype(np.float64)
        Xref = omlp.features(coarse, j, U_MAX)
        # bf16 on the GPU (rounded from an FP32 difference): within one bf16
        # ulp (2^-7 of the value at most) of the rounded oracle value
        assert np.all(np.abs(X - bf16(Xref)) <= 2.0 ** -7 * np.abs(Xref) + 1e-30)
        T = lbt.mlp_targets(d(coarse[max(j - 1, 0)]), d(coarse[j]), d(coarse[j + 1]), d(coarse[j + 2]),
                            d(fine[j * K:j * K + K + 1]), E, K, int(j == 0), U_MAX).cpu().numpy()
        Tref = omlp.targets(fine, coarse, j, K, U_MAX)
        # FP32 samples carry 2^-24 relative rounding of |u| <= u_max, i.e.
        # 2^-24 OUT_DIV in target units; fine value plus Hermite weights sum
        # to at most 4 in magnitude, and as much again for the arithmetic
        assert np.abs(T - Tref).max() <= 8 * 2.0 ** -24 * omlp.OUT_DIV
        assert np.abs(Tref).max() > 1e-4  # a residual worth learning exists


def test_forward_matches_oracle(lbt, data):
    E, fine, coarse = data
    p = omlp.init_params(3, K)
    p["b1"] = np.random.default_rng(1).normal(0, 0.1, 128)
    up = lbt.Upsampler(K=K, batch_rows=4096, master=master_vector(p))
    params = up.export()
    # both sides take the oracle's features of interval 1, rounded to bf16
    Xq = bf16(omlp.features(coarse, 1, U_MAX))
    X = torch.from_numpy(Xq).to(torch.bfloat16).contiguous().cuda()
    Y = lbt.mlp_forward(params, K, X).cpu().numpy()
    Yref, _ = omlp.forward(bf16_params(p), Xq)
    # the GPU also rounds the hidden activations to bf16 (2^-9 relative each)
    assert rel_l2(Y, Yref) <= 1e-2


def test_gradients_match_oracle(lbt, data):
    E, fine, coarse = data
    p = omlp.init_params(4, K)
    rng = np.random.default_rng(2)
    p["b1"] = rng.normal(0, 0.1, 128)
    p["b2"] = rng.normal(0, 0.1, 128)
    up = lbt.Upsampler(K=K, batch_rows=4096, master=master_vector(p))
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    j = 1
    # both sides take the oracle's features, rounded to bf16, and targets
    Xq = bf16(omlp.features(coarse, j, U_MAX))
    X = torch.from_numpy(Xq).to(torch.bfloat16).contiguous().cuda()
    T = d(omlp.targets(fine, coarse, j, K, U_MAX).astype(np.float32))
    g, loss = up.grad(X, T)
    torch.cuda.synchronize()
    gq = split_master(g.cpu().numpy(), K)
    pq = bf16_params(p)
    y, cache = omlp.forward(pq, Xq)
    gref = omlp.backward(pq, cache, y, T.cpu().numpy().astype(np.float64))
    assert abs(loss.item() - omlp.loss(y, T.cpu().numpy().astype(np.float64))) <= 2e-2 * omlp.loss(y, T.cpu().numpy())
    for name in gref:
        assert rel_l2(gq[name], gref[name]) <= 1e-2, name


def _dataset(lbt, seeds, E, nint):
    # intervals 0 .. nint-1 of every seed (interval 0: clamped j-1 sample and
    # the one-sided Hermite tangent, as the step uses them)
    from paper_0809_4958_gb300 import inputs
    Xs, Ts = [], []
    for sd in seeds:
        modes = inputs.mode_table(sd, 128, 1.0, E / 2.0, E)
        fine = lbt.synth_faces(modes, E, 1, 0, (nint + 2) * K + 1, torch.float32)
        coarse = fine[::K]
        for j in range(0, nint):
            jm = max(j - 1, 0)
            Xs.append(lbt.mlp_features(coarse[jm], coarse[j], coarse[j + 1], coarse[j + 2], E, U_MAX))
            Ts.append(lbt.mlp_targets(coarse[jm], coarse[j], coarse[j + 1], coarse[j + 2],
                                      fine[j * K:j * K + K + 1].contiguous(), E, K, int(j == 0), U_MAX))
    return torch.cat(Xs), torch.cat(Ts)


def train(lbt, X, T, steps, lr=2e-3, batch=8192, seed=0):
    # Adam with a cosine learning-rate decay
    from paper_0809_4958_gb300 import inputs
    up = lbt.Upsampler(K=K, batch_rows=batch, master=inputs.mlp_init(seed, K))
    gen = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (batch,), device="cuda", generator=gen)
        up.step(X[idx].contiguous(), T[idx].contiguous(), lr * 0.5 * (1.0 + np.cos(np.pi * it / steps)))
        if it % 50 == 0 or it == steps - 1:
            losses.append(up.loss.item())
    return up, losses


def test_training_reduces_the_loss(lbt):
    X, T = _dataset(lbt, [31, 32], 16, 6)
    up, losses = train(lbt, X, T, 300)
    assert losses[-1] < 0.5 * losses[0], losses


def test_zero_network_is_hermite_inside_the_step(lbt):
    zero = np.zeros(32 * 128 + 128 + 128 * 128 + 128 + 128 * 3 * K + 3 * K, np.float32)
    up = lbt.Upsampler(K=K, batch_rows=256, master=zero)
    params = up.export()
    c_h = Case(16, 0.8, 64, M=32, K=K, time_interp=1, nbeads=6)
    c_m = Case(16, 0.8, 64, M=32, K=K, time_interp=2, nbeads=6)
    rh = GpuRunner(lbt, torch, [c_h], 1)
    rm = GpuRunner(lbt, torch, [c_m], 1)
    rm.tr.lb_mlp_bind(params, U_MAX)
    rh.step(64)
    rm.step(64)
    assert np.array_equal(rh.tr.deviations(0), rm.tr.deviations(0))


def test_mlp_boundary_matches_oracle(lbt):
    # a network with non-zero weights: the GPU step with its bf16 residual
    # against the oracle step with the FP64 residual of the same weights
    E = 16
    p = omlp.init_params(7, K, scale=0.3)
    p["b3"] = np.random.default_rng(3).normal(0, 1.0, 3 * K)
    up = lbt.Upsampler(K=K, batch_rows=256, master=master_vector(p))
    params = up.export()
    c = Case(E, 0.8, 64, M=32, K=K, time_interp=2)
    resid = np.stack([omlp.residual_block(bf16_params(p), c.samples, j, K, U_MAX) for j in range(64 // K)])
    sim = oracle.Sim(c.oracle_box(), c.u0, c.samples, resid=resid)
    assert sim.run(64) == 0
    r = GpuRunner(lbt, torch, [c], 1)
    r.tr.lb_mlp_bind(params, U_MAX)
    r.step(64)
    u = r.tr.fields(0)[1]
    u_ref = sim.fields()[1]
    herm = Case(E, 0.8, 64, M=32, K=K, time_interp=1).run_oracle().fields()[1]
    assert rel_l2(interior(u_ref), interior(herm)) > 1e-3  # the residual matters
    assert rel_l2(interior(u), interior(u_ref)) <= 2e-3


def test_learned_boundary_beats_hermite(lbt):
    # train on boundary data of some boxes, then on held-out boxes with samples
    # every K = 16 steps: (1) the boundary residual the network leaves, against
    # the residual of Hermite alone; (2) the interior velocity error against
    # the run that sees the boundary every step, Hermite vs Hermite + network
    E = 16
    X, T = _dataset(lbt, list(range(41, 53)), E, 8)
    up, losses = train(lbt, X, T, 2500)
    params = up.export()
    Xh, Th = _dataset(lbt, [91, 92], E, 8)
    Yh = lbt.mlp_forward(params, K, Xh)
    ratio = float(((Yh - Th) ** 2).mean() / (Th ** 2).mean())
    print("held-out boundary residual left by the network: %.3f of Hermite's" % ratio)
    assert ratio < 0.5
    errs = {"hermite": [], "mlp": []}
    for sd in (91, 92):
        ref = Case(E, 0.8, 128, seed=sd, M=128, K=1, time_interp=0)
        rr = GpuRunner(lbt, torch, [ref], 1)
        rr.step(128)
        u_ref = rr.tr.fields(0)[1]
        for name, ti in (("hermite", 1), ("mlp", 2)):
            c = Case(E, 0.8, 128, seed=sd, M=128, K=K, time_interp=ti)
            r = GpuRunner(lbt, torch, [c], 1)
            if ti == 2:
                r.tr.lb_mlp_bind(params, U_MAX)
            r.step(128)
            errs[name].append(rel_l2(interior(r.tr.fields(0)[1]), interior(u_ref)))
    print("interior velocity error vs every-step boundary: hermite %s, learned %s" % (errs["hermite"], errs["mlp"]))
    assert np.mean(errs["mlp"]) < np.mean(errs["hermite"])
