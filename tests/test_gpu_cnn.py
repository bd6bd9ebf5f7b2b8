"""GPU parity of the residual CNN prox against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import cnn
from synth.cnn_init import init_params

pytestmark = pytest.mark.gpu


def _sparse_exact_params(seed):
    """Every output channel of every layer reads one or two (tap, channel)
    pairs with power-of-two weights and zero bias: each sum has at most two
    terms and is exact in float32 and float64 alike, so both sides round the
    same exact value to bfloat16 and the results must agree bit for bit.
    Any wrong tap, channel or operand layout shows as a mismatch."""
    g = np.random.default_rng(seed)
    parts = []
    for l in range(1, cnn.N_LAYERS + 1):
        cin, cout = cnn.CHANNELS[l - 1], cnn.CHANNELS[l]
        W = np.zeros((cout, cin, 3, 3))
        for o in range(cout):
            for _ in range(1 if l == 1 else 2):
                W[o, g.integers(cin), g.integers(3), g.integers(3)] = g.choice([0.5, 1.0, 2.0, -1.0, 0.25])
        parts += [W.ravel(), np.zeros(cout)]
    return np.concatenate(parts).astype(np.float32)


def _integer_params(seed, density=0.1):
    """Dense-ish integer network: weights in {-1, 0, 1} (about 29 non-zero
    per output channel), integer biases, integer inputs.  Every sum is an
    integer below 2^24 (checked on the oracle: at most ~2e5), hence exact in
    float32; bfloat16 rounding of integers gives integers, so both sides round
    the same exact values and must agree bit for bit while all 18 K-steps of
    every tensor-core layer contribute."""
    g = np.random.default_rng(seed)
    parts = []
    for l in range(1, cnn.N_LAYERS + 1):
        cin, cout = cnn.CHANNELS[l - 1], cnn.CHANNELS[l]
        W = g.choice([-1.0, 0.0, 1.0], size=(cout, cin, 3, 3), p=[density / 2, 1 - density, density / 2])
        parts += [W.ravel(), g.integers(-2, 3, cout).astype(float)]
    return np.concatenate(parts).astype(np.float32)


def _dense_params(seed):
    p = init_params(seed).astype(np.float64)
    g = np.random.default_rng(seed + 1)
    k = 0
    for l, (ws, bs) in enumerate(cnn.param_shapes()):
        nw = int(np.prod(ws))
        if l == cnn.N_LAYERS - 1:
            p[k:k + nw] *= 10.0                      # a residual branch of the same order as z
        p[k + nw:k + nw + bs[0]] = 0.05 * g.standard_normal(bs[0])
        k += nw + bs[0]
    return p.astype(np.float32)


def _run(params, z):
    import paper_1306_1392_b300 as P
    dev = torch.device("cuda:0")
    out = P.pyhst_cnn_forward(torch.from_numpy(params).to(dev), torch.from_numpy(z).to(dev))
    torch.cuda.synchronize()
    assert P.pyhst_device_status() == 0
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,h,w", [(1, 8, 8), (2, 37, 300), (1, 4, 128), (3, 5, 7), (1, 1, 1), (1, 130, 257)])
def test_sparse_network_is_bit_exact(n, h, w):
    params = _sparse_exact_params(100 + h + w)
    g = np.random.default_rng(h * 1000 + w)
    z = g.integers(0, 64, (n, h, w)).astype(np.float32) / 8.0
    out = _run(params, z)
    for i in range(n):
        ref, _, _ = cnn.forward(params, z[i], rounding=True)
        np.testing.assert_array_equal(out[i], ref)


@pytest.mark.parametrize("seed,n,h,w", [(0, 1, 37, 150), (4, 2, 64, 300), (2, 3, 264, 384)])
def test_integer_network_is_bit_exact(seed, n, h, w):
    """The last case has 297 tiles of 8 rows x 128 pixels, more than two per
    SM, so every stage of the pipelined tensor-core kernel (double-buffered
    loads and accumulators, mbarrier phases beyond the first) is exercised."""
    params = _integer_params(seed)
    z = np.random.default_rng(seed).integers(0, 8, (n, h, w)).astype(np.float32)
    out = _run(params, z)
    for i in range(n):
        ref, _, pres = cnn.forward(params, z[i], rounding=True)
        assert max(np.abs(p).max() for p in pres) < 2 ** 24
        np.testing.assert_array_equal(out[i], ref)


@pytest.mark.parametrize("n,h,w", [(2, 64, 96), (1, 131, 260)])
def test_dense_network_within_bf16_rounding(n, h, w):
    """Random dense weights: float32 sums (tensor cores) and float64 sums
    (oracle) round to the same bfloat16 activation except when a sum falls
    within its float32 error of a rounding boundary (about 1e-5 of the
    activations); such a flip moves one activation by one bf16 unit and
    spreads through the later layers.  Perturbing the oracle's sums by
    6e-8 relative (float32-sized) moves the residual branch r = out - z by
    0.6e-3 .. 2.5e-3 relative L2 on this input.  Bound: r within 1e-2 and out
    within 2e-3 relative L2 of the oracle; a dropped K-step or tap would be
    O(1)."""
    params = _dense_params(7)
    g = np.random.default_rng(8)
    yy, xx = np.mgrid[0:h, 0:w]
    z = (0.5 + 0.3 * np.sin(xx / 7.0) * np.cos(yy / 5.0) + 0.05 * g.standard_normal((n, h, w))).astype(np.float32)
    out = _run(params, z)
    for i in range(n):
        ref, _, _ = cnn.forward(params, z[i], rounding=True)
        r_gpu, r_ref = out[i] - z[i], ref - z[i]
        assert np.linalg.norm(r_ref) > 0.05 * np.linalg.norm(z[i])     # the branch is not negligible
        assert np.linalg.norm(r_gpu - r_ref) <= 1e-2 * np.linalg.norm(r_ref)
        assert np.linalg.norm(out[i] - ref) <= 2e-3 * np.linalg.norm(ref)


def test_trained_network_full_size_sampled():
    """The configuration the learned solve runs: the trained weights on a
    64 x 512^2 stack.  Each output pixel depends on z within 8 pixels (eight
    3 x 3 layers; the oracle pin test_receptive_field_is_eight_pixels), so
    the oracle runs the network on the 17 x 17 crop around each sampled pixel
    (or the part of it inside the image) and gives the full image's value.
    Same bounds as the dense test, over the samples."""
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    params = np.load(os.path.join(root, "paper_1306_1392_b300", "weights", "prox_cnn_foam512.npy")).astype(np.float32)
    n, h, w = 64, 512, 512
    g = np.random.default_rng(12)
    yy, xx = np.mgrid[0:h, 0:w]
    base = 0.5 + 0.3 * np.sin(xx / 23.0) * np.cos(yy / 17.0)
    z = (base[None] + 0.05 * g.standard_normal((n, h, w))).astype(np.float32)
    out = _run(params, z)
    pts = list(zip(g.integers(0, n, 120), g.integers(0, h, 120), g.integers(0, w, 120)))
    pts += [(0, 0, 0), (1, h - 1, w - 1), (2, 0, w - 1), (63, h - 1, 0), (5, 127, 128), (6, 255, 256)]
    rg, rr, og, orf = [], [], [], []
    for s_, i, j in pts:
        i0, i1, j0, j1 = max(0, i - 8), min(h, i + 9), max(0, j - 8), min(w, j + 9)
        ref, _, _ = cnn.forward(params, z[s_, i0:i1, j0:j1], rounding=True)
        v = ref[i - i0, j - j0]
        og.append(out[s_, i, j]); orf.append(v)
        rg.append(out[s_, i, j] - z[s_, i, j]); rr.append(v - z[s_, i, j])
    rg, rr, og, orf = (np.asarray(a, np.float64) for a in (rg, rr, og, orf))
    assert np.linalg.norm(rg - rr) <= 1e-2 * np.linalg.norm(rr)
    assert np.linalg.norm(og - orf) <= 2e-3 * np.linalg.norm(orf)


def test_forward_rejects_bad_arguments():
    import paper_1306_1392_b300 as P
    from paper_1306_1392_b300 import _lib as L
    dev = torch.device("cuda:0")
    p = torch.zeros(P.pyhst_cnn_param_count(), device=dev)
    z = torch.zeros((1, 8, 8), device=dev)
    assert L.lib.pyhst_cnn_forward(p.data_ptr(), z.data_ptr(), z.data_ptr(), 0, 8, 8, None, 0, None) == -1
    ws = torch.empty(16, dtype=torch.uint8, device=dev)
    assert L.lib.pyhst_cnn_forward(p.data_ptr(), z.data_ptr(), z.data_ptr(), 1, 8, 8, ws.data_ptr(), 16, None) == -3


def _layer_slices():
    k, out = 0, []
    for ws, bs in cnn.param_shapes():
        nw, nb = int(np.prod(ws)), bs[0]
        out.append(slice(k, k + nw + nb))
        k += nw + nb
    return out


def test_gradient_matches_oracle_chain_rule():
    """Batch of two 24 x 40 images (ragged against the 8 x 32 gradient
    tiles and the 128-pixel convolution strips).  The GPU keeps the gradients
    of hidden pre-activations in bf16 (2^-9 relative rounding each) and sums
    in float32; the oracle differentiates the same bf16 network in FP64.
    Bound per layer: relative L2 <= 2e-2 and cosine >= 0.999; a wrong tap,
    channel or transpose would give an O(1) error."""
    import paper_1306_1392_b300 as P
    params = _dense_params(11)
    g = np.random.default_rng(12)
    n, h, w = 2, 24, 40
    yy, xx = np.mgrid[0:h, 0:w]
    z = (0.5 + 0.3 * np.sin(xx / 5.0) * np.cos(yy / 4.0) + 0.05 * g.standard_normal((n, h, w))).astype(np.float32)
    t = (z + 0.1 * g.standard_normal((n, h, w))).astype(np.float32)
    dev = torch.device("cuda:0")
    grad, loss = P.pyhst_cnn_grad(torch.from_numpy(params).to(dev), torch.from_numpy(z).to(dev),
                                  torch.from_numpy(t).to(dev))
    torch.cuda.synchronize()
    assert P.pyhst_device_status() == 0
    grad = grad.cpu().numpy().astype(np.float64)
    ref_l, ref_g = 0.0, np.zeros(params.size)
    for i in range(n):
        li, gi = cnn.loss_and_grad(params, z[i], t[i], rounding=True)
        ref_l += li / n
        ref_g += gi / n
    assert loss.item() == pytest.approx(ref_l, rel=2e-3)
    for sl in _layer_slices():
        a, b = grad[sl], ref_g[sl]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b), sl
        assert np.vdot(a, b) >= 0.999 * np.linalg.norm(a) * np.linalg.norm(b), sl


def test_adam_matches_oracle_and_descends():
    import paper_1306_1392_b300 as P
    dev = torch.device("cuda:0")
    g = np.random.default_rng(13)
    npar = P.pyhst_cnn_param_count()
    p0 = g.standard_normal(npar).astype(np.float32)
    gr = g.standard_normal(npar).astype(np.float32)
    m0 = (0.1 * g.standard_normal(npar)).astype(np.float32)
    v0 = (0.01 * g.uniform(0, 1, npar)).astype(np.float32)
    pt, mt, vt = (torch.from_numpy(a.copy()).to(dev) for a in (p0, m0, v0))
    P.pyhst_cnn_adam(pt, torch.from_numpy(gr).to(dev), mt, vt, 3, 1e-3)
    # the kernel computes with the float32 values of lr, beta1, beta2, eps; the
    # oracle takes the same values and sums exactly
    f = lambda a: float(np.float32(a))
    rp, rm, rv = cnn.adam_step(p0.astype(np.float64), gr.astype(np.float64), m0.astype(np.float64),
                               v0.astype(np.float64), 3, f(1e-3), f(0.9), f(0.999), f(1e-8))
    # two-term float32 sums: within a few units of 2^-24 of the operands
    ulp = 2.0 ** -24
    b1, b2 = f(0.9), f(0.999)
    assert np.all(np.abs(mt.cpu().numpy() - rm) <= 4 * ulp * (b1 * np.abs(m0) + (1 - b1) * np.abs(gr)))
    assert np.all(np.abs(vt.cpu().numpy() - rv) <= 4 * ulp * (b2 * v0 + (1 - b2) * gr.astype(np.float64) ** 2))
    # the new parameter: one float32 rounding of p plus 1e-4 of the step
    assert np.all(np.abs(pt.cpu().numpy() - rp) <= 2.0 ** -23 * np.abs(p0) + 1e-4 * np.abs(rp - p0))
    # a few steps on one batch lower its loss
    params = torch.from_numpy(init_params(3)).to(dev)
    z = torch.rand((2, 32, 48), device=dev)
    t = z + 0.1 * torch.sin(torch.arange(48, device=dev) / 3.0)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    losses = []
    for k in range(1, 21):
        grad, loss = P.pyhst_cnn_grad(params, z, t)
        losses.append(loss.item())
        P.pyhst_cnn_adam(params, grad, m, v, k, 1e-3)
    assert losses[-1] < 0.9 * losses[0]


def test_pnp_solve_matches_oracle():
    """FISTA with the network as prox, 3 iterations on a 48^2 foam with 16
    angles, against the oracle's plug-and-play FISTA with the same L.  The
    network's bf16 rounding flips (see the dense test) are the only source of
    difference beyond float32 rounding: bound 5e-3 relative L2."""
    import oracle as orc
    import paper_1306_1392_b300 as P
    from synth import acquisition as acq
    dev = torch.device("cuda:0")
    fs = acq.foam_slice(48, 16, seed=9, truth=False)
    geo = P.Geometry(fs.angles.to(dev), fs.axis.to(dev), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    og = orc.Geometry(fs.angles.double().numpy(), fs.axis.double().numpy(), fs.n_bins, fs.nx, fs.ny, fs.pixel_size)
    L = 1.01 * orc.power_iteration(og, np.ones((fs.ny, fs.nx)), 30)[0]
    params = init_params(21)
    sino = fs.extra["sino"]
    x, e, lip = P.pyhst_pnp_solve(geo, sino.to(dev), torch.from_numpy(params).to(dev),
                                  P.TvOptions(beta=0.0, n_iter=3, lipschitz=L))
    torch.cuda.synchronize()
    assert P.pyhst_device_status() == 0
    xr, er = cnn.pnp_fista(og, sino.double().numpy(), params, L, 3)
    xg = x[0].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xr) <= 5e-3 * np.linalg.norm(xr)
    np.testing.assert_allclose(e[0].cpu().numpy(), er, rtol=1e-2)


def test_wait_give_up_is_reported_and_the_next_call_succeeds():
    """Failure detection without a GPU fault.  With the tensor-core kernels'
    pipeline waits set to give up without polling, the first wait of a
    16 x 256^2 forward pass runs out: the kernel stops issuing
    work, drains the tensor-core operations it already issued (that wait keeps
    the default limit), frees its tensor memory and returns, and the device
    status word carries bit 1.  With the default limit restored, the next
    call is bit-exact against the oracle and sets no bit."""
    import paper_1306_1392_b300 as P
    dev = torch.device("cuda:0")
    params = _integer_params(7)
    pd = torch.from_numpy(params).to(dev)
    g = np.random.default_rng(7)
    zbig = torch.from_numpy(g.integers(0, 8, (16, 256, 256)).astype(np.float32)).to(dev)
    P.pyhst_device_status(clear=True)
    hit = 0
    try:
        P.pyhst_set_wait_limit(0)
        for _ in range(2):
            P.pyhst_cnn_forward(pd, zbig)
            torch.cuda.synchronize()
            hit |= P.pyhst_device_status(clear=True)
            if hit:
                break
    finally:
        P.pyhst_set_wait_limit(-1)
    assert hit & 1
    z = g.integers(0, 8, (1, 40, 200)).astype(np.float32)
    out = _run(params, z)                       # asserts the status word is clear again
    ref, _, _ = cnn.forward(params, z[0], rounding=True)
    np.testing.assert_array_equal(out[0], ref)


def test_learned_prox_study_runs_small(cuda_device):
    """The benchmark's learned-prox study end to end at a small size (2
    held-out foams, short solves, one point of every grid): every solve is
    timed and scored, and the equal-PSNR summary, when a learned solve
    reaches the target, compares like with like."""
    import os
    from paper_1306_1392_b300 import train_prox
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    params = torch.from_numpy(np.load(os.path.join(root, "paper_1306_1392_b300", "weights",
                                                   "prox_cnn_foam512.npy")).astype(np.float32)).to(cuda_device)
    r = train_prox.evaluate(params, cuda_device, n_eval=2, ks=(1,), n_iter_tv=20, tv_long=0, hybrid_kt=(10,),
                            tv_first=(8,), learned_steps=(2,), tv_zero=(15,), tv_warm_dual=((5, 15),),
                            learned_warm_dual=((5, 8, 2),))
    variants = {x["variant"] for x in r["pnp"]}
    assert {"ista", "fbp+tv", "tv+ista2", "tv", "tv-warm-dual5", "tv-warm-dual5+ista2"} <= variants
    assert all(x["s_per_slice"] > 0 and np.isfinite(x["psnr_mean"]) for x in r["pnp"])
    e = r["equal_psnr"]
    if e is not None:
        assert "warm-dual" not in e["pnp_variant"] and "warm-dual" not in e["tv_variant"]
        assert e["speedup"] == e["tv_s_per_slice"] / e["pnp_s_per_slice"]
        assert e["any_tv_s_per_slice"] <= e["tv_s_per_slice"] and e["any_pnp_s_per_slice"] <= e["pnp_s_per_slice"]
