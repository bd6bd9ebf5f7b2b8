"""Train the residual CNN prox on pairs that the method itself generates,
and measure it in the plug-and-play loop against the plain TV solve.

Pairs.  Each seeded phantom (512^2, Voronoi foam or random ellipses, 100
angles over 180 degrees, Poisson counts at 1e4 photons per bin) is
reconstructed by FISTA-TV (Eq. 3; beta 1.78e-3, 20 Chambolle steps) for 1000
iterations with pyhst_tv_solve_capture, started from its filtered
back-projection.  The 1000th iterate is the target; the prox inputs z_k of
the same run at the capture iterations are the network inputs (one pair per
capture iteration).  The learned solve starts from the FBP as well, so the
network sees gradient steps taken near the solution, as in its own loop.

The learned solve.  FBP, then K_T FISTA-TV iterations from it, then K_L
ISTA iterations whose prox is the network (pyhst_pnp_solve): TV removes the
FBP's noise and streaks, the network takes the slow tail of the TV
convergence in one or two steps.

Training.  Adam on the mean squared error over random 128^2 crops (random
flips and transposes), through pyhst_cnn_grad / pyhst_cnn_adam.  Then, for
a few rounds, the current network runs the learned solve on the training
sinograms (K_T in LOOP_TV); the gradient-step outputs z it meets become
further inputs for the same targets, and training continues, so that the
network sees the inputs of its own iteration.

Evaluation.  On held-out seeded foams: the plain TV solve (200 FISTA
iterations x 20 Chambolle steps from zero) and FBP followed by
pyhst_pnp_solve for several iteration counts K, each timed end to end with
CUDA events; PSNR over the inscribed disk against the phantom.

    python -m paper_1306_1392_b300.train_prox --out paper_1306_1392_b300/weights/prox_cnn_foam512.npy
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

N, N_ANGLES, PHOTONS, BETA = 512, 100, 1e4, 1.7783e-3
CAPTURE = (10, 15, 20, 25, 30, 40, 50)
LOOP_TV = (20, 30, 40)          # TV iterations before the learned steps, in the training rounds
LEARNED_STEPS = 2               # learned ISTA steps after the TV iterations
TRAIN_SEED0, EVAL_SEED0 = 200000, 300000


def psnr(x: np.ndarray, truth: np.ndarray) -> float:
    """PSNR over the inscribed disk r <= N/2 - 1, peak = truth range."""
    n = truth.shape[0]
    yy, xx = np.meshgrid(np.arange(n) - (n - 1) / 2, np.arange(n) - (n - 1) / 2, indexing="ij")
    m = np.hypot(xx, yy) <= n / 2 - 1
    mse = float(np.mean((x[m] - truth[m]) ** 2))
    return 10 * math.log10((truth.max() - truth.min()) ** 2 / mse)


def phantom(seed: int, dev, truth: bool):
    from synth import acquisition as acq
    if seed % 2 == 0:
        return acq.foam_slice(N, N_ANGLES, seed=seed, photons=PHOTONS, device=dev, truth=truth)
    return acq.ellipse_slice(N, N_ANGLES, seed=seed, photons=PHOTONS, device=dev, truth=truth)


def geometry(dev):
    from synth import acquisition as acq
    from . import Geometry
    ang = acq.uniform_angles(N_ANGLES)
    return Geometry(ang.to(dev), torch.full((N_ANGLES,), (N - 1) / 2.0, device=dev), N, N, N, 2.0 / N)


def step_size(geo, dev) -> float:
    from . import TvOptions, pyhst_tv_solve
    sino = torch.zeros((1, N_ANGLES, N), device=dev)
    _, _, lip = pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=1, n_inner=1, n_power_iter=50), energy=False)
    return float(lip[0].item())


def training_sinograms(c0: int, c1: int, dev):
    return torch.stack([phantom(TRAIN_SEED0 + k, dev, False).extra["sino"].to(dev) for k in range(c0, c1)]).contiguous()


def generate_pairs(n_phantoms: int, dev, chunk: int = 64, n_iter: int = 1000, log=print, capture=CAPTURE):
    """inputs [n_phantoms, len(CAPTURE), N, N], targets [n_phantoms, N, N]
    (device float32)."""
    from . import TvOptions, pyhst_fbp, pyhst_tv_solve_capture
    geo = geometry(dev)
    L = step_size(geo, dev)
    inputs = torch.empty((n_phantoms, len(capture), N, N), device=dev)
    targets = torch.empty((n_phantoms, N, N), device=dev)
    opts = TvOptions(beta=BETA, n_iter=n_iter, n_inner=20, lipschitz=L, warm_start=True)
    t0 = time.time()
    for c0 in range(0, n_phantoms, chunk):
        c1 = min(n_phantoms, c0 + chunk)
        sino = training_sinograms(c0, c1, dev)
        x0 = pyhst_fbp(geo, sino, "f32_sino")
        x, cap = pyhst_tv_solve_capture(geo, sino, opts, capture, x=x0)
        targets[c0:c1] = x
        inputs[c0:c1] = cap.permute(1, 0, 2, 3)
        log(f"pairs {c1}/{n_phantoms}  {time.time() - t0:.1f} s")
    return inputs, targets, L


def loop_inputs(params, n_phantoms: int, K: int, L: float, dev, chunk: int = 64):
    """The prox inputs z of the learned solve on the training sinograms, for
    K_T in LOOP_TV and K learned steps each: [n_phantoms, len(LOOP_TV) K, N, N]."""
    from . import TvOptions, pyhst_cnn_forward, pyhst_fbp, pyhst_tv_solve
    geo = geometry(dev)
    out = torch.empty((n_phantoms, len(LOOP_TV) * K, N, N), device=dev)
    step = TvOptions(beta=0.0, n_iter=1, lipschitz=L, warm_start=True, use_fista=False)
    for c0 in range(0, n_phantoms, chunk):
        c1 = min(n_phantoms, c0 + chunk)
        sino = training_sinograms(c0, c1, dev)
        fbp = pyhst_fbp(geo, sino, "f32_sino")
        for j, kt in enumerate(LOOP_TV):
            x, _, _ = pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=kt, n_inner=20, lipschitz=L,
                                                          warm_start=True), x=fbp.clone(), energy=False)
            for k in range(K):
                z, _, _ = pyhst_tv_solve(geo, sino, step, x=x.clone(), energy=False)   # z = x - (1/L) P^T (P x - y)
                out[c0:c1, j * K + k] = z
                x = pyhst_cnn_forward(params, z)
    return out


def train(inputs, targets, steps: int, batch: int = 16, crop: int = 128, lr: float = 1e-3, seed: int = 1,
          log=print, log_every: int = 500, params=None):
    from synth.cnn_init import init_params
    from . import pyhst_cnn_adam, pyhst_cnn_grad
    dev = inputs.device
    g = torch.Generator(device="cpu").manual_seed(seed)
    params = torch.from_numpy(init_params(seed)).to(dev) if params is None else params.clone()
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    n_ph, n_cap = inputs.shape[0], inputs.shape[1]
    zb = torch.empty((batch, crop, crop), device=dev)
    tb = torch.empty_like(zb)
    ws = None
    hist = []
    acc = torch.zeros((), dtype=torch.float64, device=dev)
    for step in range(1, steps + 1):
        p = torch.randint(0, n_ph, (batch,), generator=g)
        k = torch.randint(0, n_cap, (batch,), generator=g)
        oy = torch.randint(0, N - crop + 1, (batch,), generator=g)
        ox = torch.randint(0, N - crop + 1, (batch,), generator=g)
        aug = torch.randint(0, 8, (batch,), generator=g)
        for b in range(batch):
            zi = inputs[p[b], k[b], oy[b]:oy[b] + crop, ox[b]:ox[b] + crop]
            ti = targets[p[b], oy[b]:oy[b] + crop, ox[b]:ox[b] + crop]
            a = int(aug[b])
            if a & 1:
                zi, ti = zi.flip(0), ti.flip(0)
            if a & 2:
                zi, ti = zi.flip(1), ti.flip(1)
            if a & 4:
                zi, ti = zi.t(), ti.t()
            zb[b] = zi
            tb[b] = ti
        if ws is None:
            from . import _lib as L
            ws = torch.empty(L.lib.pyhst_cnn_train_workspace_size(batch, crop, crop), dtype=torch.uint8, device=dev)
        grad, loss = pyhst_cnn_grad(params, zb, tb, workspace=ws)
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps))      # cosine decay
        pyhst_cnn_adam(params, grad, m, v, step, max(lr_t, 1e-6))
        acc += loss[0]
        if step == 1 or step % log_every == 0 or step == steps:
            span = 1 if step == 1 else (step % log_every or log_every)
            hist.append((step, acc.item() / span))                  # mean loss since the last report
            acc.zero_()
            log(f"step {step}  loss {hist[-1][1]:.4e}  lr {lr_t:.2e}")
    return params, hist


def equal_psnr(rows, target, s_target):
    """Time to the target PSNR, from measured solves.  rows: dicts with
    variant, n_iter, s_per_slice, psnr_mean.  Plain TV variants are "tv"
    (from zero), "fbp+tv" (from the FBP) and "tv-warm-dual<n>" (warm-started
    proxes); every other variant is a learned solve, warm-started when its
    name holds "warm-dual".  Each ratio compares like with like:
    ``speedup``, the fastest solves reaching the target whose proxes all
    start from a zero dual field (the paper's prox); ``speedup_vs_any_tv``,
    the fastest with warm-started proxes allowed on both sides;
    ``speedup_vs_tv_from_zero``, against s_target, the solve that sets the
    target.  None when no learned solve reaches the target."""
    is_cold = lambda v: "warm-dual" not in v          # every prox from a zero dual field
    is_plain = lambda v: v in ("tv", "fbp+tv") or (v.startswith("tv-warm-dual") and "+" not in v)
    fastest = lambda rs: min((r for r in rs if r["psnr_mean"] >= target), key=lambda r: r["s_per_slice"],
                             default=None)
    plain = [r for r in rows if is_plain(r["variant"])]
    learned = [r for r in rows if not is_plain(r["variant"])]
    tv_cold, tv_any = fastest([r for r in plain if is_cold(r["variant"])]), fastest(plain)
    ln_cold, ln_any = fastest([r for r in learned if is_cold(r["variant"])]), fastest(learned)
    if not (tv_cold and ln_cold and tv_any and ln_any):
        return None
    return {"target_psnr": target, "pnp_variant": ln_cold["variant"], "pnp_n_iter": ln_cold["n_iter"],
            "pnp_s_per_slice": ln_cold["s_per_slice"], "pnp_psnr": ln_cold["psnr_mean"],
            "tv_variant": tv_cold["variant"], "tv_n_iter": tv_cold["n_iter"],
            "tv_s_per_slice": tv_cold["s_per_slice"], "tv_psnr": tv_cold["psnr_mean"],
            "speedup": tv_cold["s_per_slice"] / ln_cold["s_per_slice"],
            "any_pnp_variant": ln_any["variant"], "any_pnp_n_iter": ln_any["n_iter"],
            "any_pnp_s_per_slice": ln_any["s_per_slice"], "any_pnp_psnr": ln_any["psnr_mean"],
            "any_tv_variant": tv_any["variant"], "any_tv_n_iter": tv_any["n_iter"],
            "any_tv_s_per_slice": tv_any["s_per_slice"], "any_tv_psnr": tv_any["psnr_mean"],
            "speedup_vs_any_tv": tv_any["s_per_slice"] / ln_any["s_per_slice"],
            "speedup_vs_tv_from_zero": s_target / ln_cold["s_per_slice"]}


def evaluate(params, dev, n_eval: int = 64, ks=(1, 2, 3, 5), n_iter_tv: int = 200,
             L: float = None, variants=(("ista", False),), tv_long: int = 1000,
             hybrid_kl=(0,), hybrid_kt=(30, 40, 50, 75, 100), tv_first=(20, 25, 30, 35, 40),
             learned_steps=(1, 2), tv_zero=(), tv_warm_dual=(), learned_warm_dual=()):
    """Plain TV vs the learned prox on held-out seeded foams (even seeds).
    The target PSNR is plain TV's after n_iter_tv iterations from zero.  The
    learned solve is FBP, K_T FISTA-TV iterations (tv_first), then K_L ISTA
    steps with the network as the prox (learned_steps); the fastest (K_T, K_L)
    whose mean PSNR reaches the target is compared (equal_psnr) with the
    fastest plain TV solve that reaches it: from zero with n_iter_tv or fewer
    (tv_zero) iterations, from the FBP (hybrid_kt with K_L = 0), or from zero
    with (n_inner, n_iter) of tv_warm_dual and each prox's dual field starting
    at the previous prox's.  learned_warm_dual: (n_inner, K_T, K_L) learned
    solves whose TV phase uses warm-started proxes of n_inner steps.
    ``speedup`` compares the fastest of each side whose proxes start from a
    zero dual field (the paper's prox), ``speedup_vs_any_tv`` the fastest of
    each side with warm-started proxes allowed."""
    from . import TvOptions, pyhst_fbp, pyhst_pnp_solve, pyhst_tv_solve
    geo = geometry(dev)
    if L is None:
        L = step_size(geo, dev)
    sl = [phantom(EVAL_SEED0 + 2 * k, dev, True) for k in range(n_eval)]
    sino = torch.stack([s.extra["sino"].to(dev) for s in sl]).contiguous()
    truth = [s.truth.double().cpu().numpy() for s in sl]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) * 1e-3

    tv_opts = TvOptions(beta=BETA, n_iter=n_iter_tv, n_inner=20, lipschitz=L)
    (x_tv, _, _), t_tv = timed(lambda: pyhst_tv_solve(geo, sino, tv_opts, energy=False))
    ps_tv = float(np.mean([psnr(x_tv[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
    res = {"workload": f"{n_eval} held-out foams {N}^2, {N_ANGLES} angles, Poisson {PHOTONS:.0e}",
           "tv": {"n_iter": n_iter_tv, "n_inner": 20, "beta": BETA, "s_per_slice": t_tv / n_eval,
                  "psnr_mean": ps_tv},
           "pnp": []}
    if tv_long:
        x_l, _, _ = pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=tv_long, n_inner=20, lipschitz=L),
                                   energy=False)
        res["tv_long"] = {"n_iter": tv_long,
                          "psnr_mean": float(np.mean([psnr(x_l[i].double().cpu().numpy(), truth[i])
                                                      for i in range(n_eval)]))}

    def learned(K, fista):
        x0 = pyhst_fbp(geo, sino, "f32_sino")
        return pyhst_pnp_solve(geo, sino, params, TvOptions(beta=0.0, n_iter=K, lipschitz=L, warm_start=True,
                                                            use_fista=fista), x=x0, energy=False)

    (x_fbp, ), _ = timed(lambda: (pyhst_fbp(geo, sino, "f32_sino"),))
    res["fbp_psnr_mean"] = float(np.mean([psnr(x_fbp[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
    for name, fista in variants:
        for K in ks:
            (x, _, _), t = timed(lambda: learned(K, fista))
            ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
            res["pnp"].append({"variant": name, "n_iter": K, "s_per_slice": t / n_eval, "psnr_mean": ps})
    # plain TV from the FBP, and the learned loop (ISTA, K_L iterations) followed by TV iterations
    def tv_from(x0, K):
        return pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=K, n_inner=20, lipschitz=L, warm_start=True),
                              x=x0, energy=False)

    def hybrid(KL, KT):
        x0 = pyhst_fbp(geo, sino, "f32_sino")
        if KL:
            x0, _, _ = pyhst_pnp_solve(geo, sino, params, TvOptions(beta=0.0, n_iter=KL, lipschitz=L, warm_start=True,
                                                                    use_fista=False), x=x0, energy=False)
        return tv_from(x0, KT) if KT else (x0, None, None)

    def tv_then_learned(KT, KL, n_in=20, warm_dual=False):
        x0 = pyhst_fbp(geo, sino, "f32_sino")
        x0, _, _ = pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=KT, n_inner=n_in, lipschitz=L,
                                                       warm_start=True, warm_dual=warm_dual), x=x0, energy=False)
        return pyhst_pnp_solve(geo, sino, params, TvOptions(beta=0.0, n_iter=KL, lipschitz=L, warm_start=True,
                                                            use_fista=False), x=x0, energy=False)

    for KL in hybrid_kl:
        for KT in hybrid_kt:
            (x, _, _), t = timed(lambda: hybrid(KL, KT))
            ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
            res["pnp"].append({"variant": f"ista{KL}+tv" if KL else "fbp+tv", "n_iter": KT,
                               "s_per_slice": t / n_eval, "psnr_mean": ps})
    for KL in learned_steps:
        for KT in tv_first:
            (x, _, _), t = timed(lambda: tv_then_learned(KT, KL))
            ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
            res["pnp"].append({"variant": f"tv+ista{KL}", "n_iter": KT, "s_per_slice": t / n_eval, "psnr_mean": ps})
    for n_in, KT, KL in learned_warm_dual:
        (x, _, _), t = timed(lambda: tv_then_learned(KT, KL, n_in, True))
        ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
        res["pnp"].append({"variant": f"tv-warm-dual{n_in}+ista{KL}", "n_iter": KT, "s_per_slice": t / n_eval,
                           "psnr_mean": ps})
    for KT in tv_zero:
        (x, _, _), t = timed(lambda: pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=KT, n_inner=20,
                                                                         lipschitz=L), energy=False))
        ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
        res["pnp"].append({"variant": "tv", "n_iter": KT, "s_per_slice": t / n_eval, "psnr_mean": ps})
    for n_in, KT in tv_warm_dual:
        (x, _, _), t = timed(lambda: pyhst_tv_solve(geo, sino, TvOptions(beta=BETA, n_iter=KT, n_inner=n_in,
                                                                         lipschitz=L, warm_dual=True), energy=False))
        ps = float(np.mean([psnr(x[i].double().cpu().numpy(), truth[i]) for i in range(n_eval)]))
        res["pnp"].append({"variant": f"tv-warm-dual{n_in}", "n_iter": KT, "s_per_slice": t / n_eval,
                           "psnr_mean": ps})
    res["equal_psnr"] = equal_psnr([{"variant": "tv", "n_iter": n_iter_tv, "s_per_slice": t_tv / n_eval,
                                      "psnr_mean": ps_tv}] + res["pnp"], ps_tv, t_tv / n_eval)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--phantoms", type=int, default=1500)
    ap.add_argument("--steps", type=int, default=16000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval", type=int, default=64)
    ap.add_argument("--rounds", type=int, default=2, help="rounds of training on the learned loop's own inputs")
    ap.add_argument("--loop-iters", type=int, default=LEARNED_STEPS)
    ap.add_argument("--round-steps", type=int, default=8000)
    ap.add_argument("--eval-only", help="evaluate these saved weights (.npy) instead of training")
    ap.add_argument("--capture", default=",".join(map(str, CAPTURE)),
                    help="TV iterations whose prox inputs are training inputs")
    ap.add_argument("--out")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    if a.eval_only:
        params = torch.from_numpy(np.load(a.eval_only).astype(np.float32)).to(dev)
        print(json.dumps(evaluate(params, dev, n_eval=a.eval)), flush=True)
        return
    t0 = time.time()
    capture = tuple(int(c) for c in a.capture.split(","))
    inputs, targets, L = generate_pairs(a.phantoms, dev, capture=capture)
    t1 = time.time()
    params, hist = train(inputs, targets, a.steps, batch=a.batch, lr=a.lr)
    rounds = []
    for r in range(a.rounds):
        z = loop_inputs(params, a.phantoms, a.loop_iters, L, dev)
        inputs = torch.cat([inputs, z], dim=1)
        del z
        params, h = train(inputs, targets, a.round_steps, batch=a.batch, lr=0.5 * a.lr, seed=100 + r, params=params)
        rounds.append(h[-1])
        print(f"round {r + 1}: {inputs.shape[1]} inputs per phantom, loss {h[-1][1]:.4e}", flush=True)
    torch.cuda.synchronize()
    t2 = time.time()
    np.save(a.out, params.cpu().numpy())
    del inputs, targets
    res = evaluate(params, dev, n_eval=a.eval, L=L)
    res.update(pairs=a.phantoms * len(capture), capture=list(capture), train_steps=a.steps, batch=a.batch,
               rounds=a.rounds, loop_iters=a.loop_iters, round_steps=a.round_steps, round_losses=rounds,
               gen_s=t1 - t0, train_s=t2 - t1, loss_history=hist)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
