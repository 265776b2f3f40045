"""Parity of the learned-initial-guess kernels with the FP64 oracle (oracle/warmstart.py),
and what the trained guess gains over the method without it.  Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import warmstart as ows
from oracle.stokes import SlabGeometry
from workloads import fourier_forcing_2d, random_vector

pytestmark = pytest.mark.gpu

import paper_2502_09159_gb300 as stmg
from paper_2502_09159_gb300.warmstart import ConvNet, WarmStart, channel_rms, scale_channels


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(a, b):
    a = a.detach().cpu().numpy().astype(np.float64) if isinstance(a, torch.Tensor) else np.asarray(a)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


GEOS = [(2, 3, 2, 1), (2, 4, 1, 2), (3, 2, 1, 1), (2, 2, 3, 0)]


@pytest.fixture(scope="module", params=GEOS, ids=["2d-n3-r2k1", "2d-n4-r1k2", "3d-n2-r1k1", "2d-n2-r3k0"])
def handle(request):
    dim, n, r, k = request.param
    g = stmg.SpaceTimeMG(dim=dim, n_cells=n, r=r, k=k, levels=[(n, r, k)], use_graphs=False, autotune=False)
    geo = SlabGeometry(dim, n, r, k, g.cfg.nu, g.cfg.T / g.cfg.n_slabs)
    yield g, geo
    g.close()


def test_cells_gather_matches_oracle(handle):
    g, geo = handle
    C = ows.n_channels(geo.dim, geo.r, geo.k)
    assert g.n_channels() == C
    x, base = random_vector(geo.size, 1), random_vector(geo.size, 2)
    inv = np.linspace(0.25, 3.0, C).astype(np.float32)
    ref = ows.cells_gather(geo, x, base, inv.astype(np.float64)).astype(np.float32)
    got = g.cells_gather(dev(x), base=dev(base), inv_scale=dev(inv, torch.float32)).cpu().numpy()
    assert np.array_equal(got, ref)                      # same FP64 arithmetic, one rounding
    plain = g.cells_gather(dev(x)).cpu().numpy()
    assert np.array_equal(plain, ows.cells_gather(geo, x).astype(np.float32))


def test_cells_scatter_add_matches_oracle(handle):
    g, geo = handle
    C = ows.n_channels(geo.dim, geo.r, geo.k)
    rng = np.random.default_rng(3)
    cells = rng.uniform(-1, 1, (geo.n ** geo.dim, C)).astype(np.float32)
    scale = rng.uniform(0.5, 2, C).astype(np.float32)
    x = random_vector(geo.size, 4)
    ref = ows.cells_scatter_add(geo, cells.astype(np.float64), x, scale.astype(np.float64))
    got = g.cells_scatter_add(dev(cells, torch.float32), dev(x), scale=dev(scale, torch.float32))
    assert rel(got, ref) < 1e-15
    # consistent tensors round-trip exactly
    y = random_vector(geo.size, 5)
    y[geo.dirichlet] = 0.0
    yc = g.cells_gather(dev(y))
    z = g.cells_scatter_add(yc, torch.zeros(geo.size, dtype=torch.float64, device="cuda"))
    assert rel(z, y.astype(np.float32).astype(np.float64)) < 1e-15


def test_extrapolate_and_pressure_mean_match_oracle(handle):
    g, geo = handle
    x = random_vector(geo.size, 6)
    assert rel(g.extrapolate(dev(x)), ows.extrapolate(geo, x)) < 1e-14
    assert rel(g.remove_pressure_mean(dev(x)), geo.remove_pressure_mean(x)) < 1e-14


NETS = [(2, 6, 7, 13, 20, 11, 4, False), (3, 12, 12, 13, 20, 11, 4, True), (2, 16, 16, 76, 64, 76, 4, True),
        (1, 5, 9, 3, 40, 90, 3, False), (2, 4, 4, 5, 0, 6, 1, True)]
NET_IDS = ["ragged-small", "ragged-tiles-bypass", "config5-channels-bypass", "wide-out", "single-layer-bypass"]


def make_case(case, seed=0):
    B, H, W, ci, hid, co, L = case[:7]
    skip = case[7] if len(case) > 7 else False
    rng = np.random.default_rng(seed)
    theta = (rng.standard_normal(ows.n_params(ci, hid, co, L, skip=skip)) * 0.3).astype(np.float32)
    x = rng.standard_normal((B, H, W, ci)).astype(np.float32)
    t = rng.standard_normal((B, H, W, co)).astype(np.float32)
    return theta, x, t, (ci, hid, co, L)


@pytest.mark.parametrize("case", NETS, ids=NET_IDS)
def test_net_forward_backward_match_oracle(case):
    theta, x, t, dims = make_case(case)
    B, H, W = case[:3]
    skip = case[7]
    net = ConvNet(H, W, dims[0], dims[2], dims[1], dims[3], max_batch=B, skip=skip)
    assert net.n_params == len(theta)
    net.set_params(dev(theta, torch.float32))
    th64, x64, t64 = theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    pred_ref, acts = ows.forward(th64, x64, *dims, skip=skip)
    pred = net.forward(dev(x, torch.float32))
    assert rel(pred, pred_ref) < 2e-5
    loss, gpred = net.mse(pred, dev(t, torch.float32))
    loss_ref, g_ref = ows.mse(pred_ref, t64)
    assert abs(loss.item() - loss_ref) <= 1e-5 * loss_ref
    assert rel(gpred, g_ref) < 2e-5
    grads = net.backward(dev(x, torch.float32), gpred)
    grads_ref = ows.backward(th64, acts, g_ref, *dims, skip=skip)
    assert rel(grads, grads_ref) < 1e-4
    net.close()


def test_indexed_batch_and_train_step_match_oracle():
    case = (3, 6, 7, 13, 20, 11, 4)
    theta, x, t, dims = make_case(case, seed=1)
    net = ConvNet(6, 7, dims[0], dims[2], dims[1], dims[3], max_batch=2)
    net.set_params(dev(theta, torch.float32))
    X, T = dev(x, torch.float32), dev(t, torch.float32)
    index = torch.tensor([2, 0], dtype=torch.int32, device="cuda")
    th64 = theta.astype(np.float64)
    pred_ref, acts = ows.forward(th64, x[[2, 0]].astype(np.float64), *dims)
    assert rel(net.forward(X, index=index), pred_ref) < 2e-5
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    net.train_step(X, T, index, 1e-3, 1, loss_out=loss)
    L_ref, g_ref = ows.mse(pred_ref, t[[2, 0]].astype(np.float64))
    grad_ref = ows.backward(th64, acts, g_ref, *dims)
    th_ref, _, _ = ows.adam_step(th64, grad_ref, np.zeros_like(th64), np.zeros_like(th64), 1, 1e-3)
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    # the first Adam step moves every parameter by ~lr sign(g); compare where |g| is not tiny
    big = np.abs(grad_ref) > 1e-3 * np.abs(grad_ref).max()
    assert np.abs(net.params().cpu().numpy()[big] - th_ref[big]).max() < 1e-6
    net.close()


def test_adam_matches_oracle():
    """Three Adam updates from the GPU's own gradients: each update agrees with the
    oracle's update of the same parameters, gradient and moments to FP32 rounding."""
    case = (1, 4, 4, 3, 5, 2, 2)
    theta, x, t, dims = make_case(case, seed=2)
    net = ConvNet(4, 4, dims[0], dims[2], dims[1], dims[3], max_batch=1)
    net.set_params(dev(theta, torch.float32))
    X, T = dev(x, torch.float32), dev(t, torch.float32)
    m = v = np.zeros(len(theta))
    for step in range(1, 4):
        _, g = net.mse(net.forward(X), T)
        gr = net.backward(X, g).cpu().numpy().astype(np.float64)
        before = net.params().cpu().numpy().astype(np.float64)
        net.adam(0.01, step)
        ref, m, v = ows.adam_step(before, gr, m, v, step, 0.01)
        assert np.abs(net.params().cpu().numpy() - ref).max() < 2e-6
    net.close()


def test_channel_rms_and_scale():
    rng = np.random.default_rng(7)
    d = rng.standard_normal((300, 37)).astype(np.float32)
    d[:, 5] = 0.0
    rms, inv = channel_rms(dev(d, torch.float32), 37)
    ref = ows.channel_rms(d)
    assert rel(rms, ref) < 1e-6
    assert inv[5].item() == 0.0
    s = dev(rng.uniform(0.5, 2, 37), torch.float32)
    D = dev(d, torch.float32)
    scale_channels(D, s)
    assert np.array_equal(D.cpu().numpy(), (d * s.cpu().numpy()[None, :]).astype(np.float32))


def test_training_is_deterministic():
    case = (4, 8, 8, 6, 12, 6, 3)
    _, x, t, dims = make_case(case, seed=3)
    X, T = dev(x, torch.float32), dev(t, torch.float32)
    out = []
    for _ in range(2):
        net = ConvNet(8, 8, 6, 6, 12, 3, max_batch=2, seed=5)
        idx = torch.tensor([[0, 1], [2, 3], [1, 3]], dtype=torch.int32, device="cuda")
        for s in range(3):
            net.train_step(X, T, idx[s], 1e-3, s + 1)
        out.append(net.params().cpu().numpy())
        net.close()
    assert np.array_equal(out[0], out[1])


def test_fresh_network_returns_zero_so_guess_is_extrapolation():
    g = stmg.SpaceTimeMG(dim=2, n_cells=4, r=2, k=1, use_graphs=False, autotune=False)
    ws = WarmStart(g, hidden=16, layers=3)
    x = dev(random_vector(g.size(0), 8))
    ws.add_pair(x, x)
    ws.fit(steps=0)
    a = ws.guess(x, "net")
    b = ws.guess(x, "extrapolate")
    assert torch.equal(a, b)
    assert ws.guess(x, "zero").abs().max().item() == 0.0
    g.close()


def test_adjoint_gather_and_dot_match_oracle(handle):
    g, geo = handle
    C = ows.n_channels(geo.dim, geo.r, geo.k)
    x = random_vector(geo.size, 13)
    s = np.linspace(0.5, 1.5, C).astype(np.float32)
    ref = ows.cells_gather_adjoint(geo, x, s.astype(np.float64)).astype(np.float32)
    got = g.cells_gather_adjoint(dev(x), scale=dev(s, torch.float32)).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
    y = random_vector(geo.size, 14)
    assert abs(g.dot(dev(x), dev(y)).item() - float(x @ y)) <= 1e-12 * np.abs(x).sum()


def test_trained_guess_reduces_iterations():
    """Drifting Fourier forcing on a 32x32 Q3/P2 mesh, DG(1), 64 slabs on [0, 1]: the
    network is trained on pairs of the first 32 solved slabs (the start-up transient, slabs
    0-3, left out) on the initial-residual ratio, then the next 32 slabs are solved from
    the zero, the extrapolated and the learned guess.  Every solve reaches the same
    tolerance; the learned guess must beat the zero guess clearly and must not lose to
    plain extrapolation."""
    n, r, k, N = 32, 2, 1, 64
    pb = fourier_forcing_2d(nu=1.0, seed_psi=4, seed_phi=5, drift=0.05 * 2 * np.pi)
    g = stmg.SpaceTimeMG(dim=2, n_cells=n, r=r, k=k, n_slabs=N, T=1.0, precond_precision="fp32")
    pts = g.forcing_points()
    ws = WarmStart(g, hidden=64, layers=4, capacity=N, seed=1)
    x_prev = g.zeros(0)
    for s in range(N // 2):
        b = g.slab_rhs(g.forcing(pb.forcing, s, pts), x_prev if s else None)
        x, info = g.solve_slab(b, ws.guess(x_prev, "extrapolate") if s else None)
        assert info["status"] == 0
        g.remove_pressure_mean(x)
        if s >= 4:
            ws.add_pair(x_prev, x)
        x_prev = x
    losses = ws.fit_residual(steps=600, batch=4, lr=1e-4, warmup=100)
    assert losses[-50:].mean() < 0.5 * losses[:10].mean()
    assert ws.residual_ratio() < 0.5                     # training pairs: residual^2 vs extrapolation
    its = {m: [] for m in WarmStart.MODES}
    res = {m: [] for m in WarmStart.MODES}
    for s in range(N // 2, N):
        b = g.slab_rhs(g.forcing(pb.forcing, s, pts), x_prev)
        sol = None
        for m in WarmStart.MODES:
            x0 = ws.guess(x_prev, m)
            res[m].append((torch.linalg.norm(g.residual(b, x0)) / torch.linalg.norm(b)).item())
            x, info = g.solve_slab(b, x0)
            assert info["status"] == 0 and info["rel_residual"] <= 1e-8
            its[m].append(info["iterations"])
            sol = x if m == "net" else sol
        x_prev = g.remove_pressure_mean(sol)
    mean = {m: float(np.mean(v)) for m, v in its.items()}
    r0 = {m: float(np.mean(v)) for m, v in res.items()}
    print("mean FGMRES iterations:", mean, "mean initial residual:", r0)
    assert mean["net"] < 0.75 * mean["zero"]
    assert mean["net"] <= mean["extrapolate"] + 0.5
    assert r0["net"] < r0["extrapolate"]
    g.close()
